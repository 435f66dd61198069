"""The oracle's pins must catch plausible mistakes in the steps they cover.

One mistake at a time is planted in a copy of the oracle's C source (a
textual replacement that must match exactly once, so this test breaks loudly
when the source moves), the copy is built into its own library with the
oracle's own compiler flags, and the pins covering that step run against it:
at least one must fail.  The planted mistakes change arithmetic only (signs,
comparisons, dropped terms, constants), never an index or a size, so no
mutant can read or write out of bounds.  The every-bounce composition lives
in Python and is mutated by replacing the function.  CPU only.
"""
import os
import shutil

import numpy as np
import pytest

import oracle
import scenes
import test_oracle_pins as P

# name, file, original text, planted text, pins (zero-argument callables)
C_MUTANTS = [
    ("PO: sinc over v' dropped", "oracle.c",
     "double amp = area * sinc(0.5 * dot3(q, up)) * sinc(0.5 * dot3(q, vp));",
     "double amp = area * sinc(0.5 * dot3(q, up));",
     [P.test_po_parallelogram_cells_use_cross_product_area,
      lambda: P.test_bistatic_plate_exact_integral_and_receiver_shadowing(40.0)]),
    ("PO: cell area as |u'| |v'| instead of |u' x v'|", "oracle.c",
     "double area = sqrt(dot3(cr, cr));",
     "double area = sqrt(dot3(up, up)) * sqrt(dot3(vp, vp));",
     [P.test_po_parallelogram_cells_use_cross_product_area]),
    ("PO: phase sign", "oracle.c",
     "double cre = cos(ph), cim = -sin(ph);",
     "double cre = cos(ph), cim = sin(ph);",
     [P.test_po_translation_phase_convention]),
    ("PO: V-polarisation sign", "oracle.c",
     "h[0][c] = -vl[c] / lv;",
     "h[0][c] = vl[c] / lv;",
     [lambda: P.test_bistatic_plate_exact_integral_and_receiver_shadowing(15.0)]),
    ("PO: u' and v' projections swapped", "oracle.c",
     "nu = dot3(nl, ul) / nk, nv = dot3(nl, vl) / nk;",
     "nu = dot3(nl, vl) / nk, nv = dot3(nl, ul) / nk;",
     [P.test_po_parallelogram_cells_use_cross_product_area,
      lambda: P.test_po_plate_pattern_textbook(25.0)]),
    ("PO: sign of k_s in q", "oracle.c",
     "q[c] = kw * (kl[c] - ks[c]);",
     "q[c] = kw * (kl[c] + ks[c]);",
     [lambda: P.test_po_plate_pattern_textbook(25.0)]),
    ("Eq. 4: reflection sign", "oracle_core.h",
     "for (int k = 0; k < 3; ++k) out[k] = a[k] - s * n[k];",
     "for (int k = 0; k < 3; ++k) out[k] = a[k] + s * n[k];",
     [P.test_trihedral_axis_triple_bounce_aperture]),
    ("Alg. 1: ties to the larger index", "oracle_core.h",
     "if (t < best) {",
     "if (t <= best) {",
     [lambda: P.test_gfb_nearest_and_tie_break("fp32")]),
    ("edge rule dropped", "oracle_core.h",
     "if (dt > tauL) return 1;",
     "if (dt > tauL && 0) return 1;",
     [P.test_edge_filter_handmade]),
    ("Eq. 22: sqrt(2) replaced by 1.5", "oracle_core.h",
     "if (s < 2.5) return (1.4142135623730951 * L) * s;",
     "if (s < 2.5) return (1.5 * L) * s;",
     [lambda: P.test_eq22_radius_values("fp64")]),
    ("Eq. 23: no overlap window", "oracle_core.h",
     "R lim = tb + r_ov;",
     "R lim = tb;",
     [lambda: P.test_eq23_overlap_select_and_blend("fp32")]),
    ("nearest hit replaced by the farthest", "oracle_core.h",
     "if (t < tb) {",
     "if (tb == (R)INFINITY || t > tb) {",
     [lambda: P.test_eq23_overlap_select_and_blend("fp32"),
      lambda: P.test_epsilon_minimum_travel("fp32")]),
    ("Eq. 23: blend weight rho instead of 1 - rho", "oracle_core.h",
     "R w = (R)1 - rho;",
     "R w = rho;",
     [lambda: P.test_eq23_overlap_select_and_blend("fp32")]),
    ("epsilon ignored on bounces", "oracle_core.h",
     "R E = (R)eps, RO = (R)r_ov;",
     "R E = (R)0, RO = (R)r_ov;",
     [lambda: P.test_epsilon_minimum_travel("fp32")]),
]


@pytest.fixture
def plant(tmp_path):
    """plant(file, old, new): build a copy of the oracle with one textual
    change and make it the oracle's library until the test ends."""
    src = os.path.dirname(oracle.__file__)
    saved = oracle._lib

    def _plant(fname, old, new):
        for f in ("oracle.c", "oracle_core.h"):
            shutil.copy(os.path.join(src, f), tmp_path / f)
        path = tmp_path / fname
        text = path.read_text()
        assert text.count(old) == 1, f"mutation site not found exactly once in {fname}: {old!r}"
        path.write_text(text.replace(old, new))
        so = str(tmp_path / f"liboracle_{abs(hash((fname, old, new)))}.so")
        oracle._compile(str(tmp_path / "oracle.c"), so)
        oracle._lib = oracle._bind(so)

    yield _plant
    oracle._lib = saved


def _failing(pins):
    caught = []
    for pin in pins:
        try:
            pin()
        except AssertionError:
            caught.append(pin)
    return caught


def test_an_unchanged_copy_passes_the_pins(plant):
    # the mechanism itself (copy, flags, binding) changes nothing
    name, fname, old, _, _ = C_MUTANTS[0]
    plant(fname, old, old)
    pins = [p for m in C_MUTANTS for p in m[4]]
    assert _failing(pins) == []


@pytest.mark.parametrize("mutant", C_MUTANTS, ids=[m[0] for m in C_MUTANTS])
def test_pins_catch_a_planted_mistake(mutant, plant):
    name, fname, old, new, pins = mutant
    plant(fname, old, new)
    assert _failing(pins), f"no pin caught: {name}"


# ----------------------------------------------------------------------------
# the every-bounce composition (Python)
# ----------------------------------------------------------------------------

def _every_bounce_variant(kind):
    def fn(view, splats, first, mb, eps, r_ov, freqs_hz, mode="fp32"):
        w = -np.asarray(view.d, np.float64)
        if kind == "receiver sign":
            w = -w
        E = 0.0
        top = mb if kind == "last bounce dropped" else mb + 1
        for b in range(1, top):
            depth = mb if kind == "full-depth trace at every b" else b
            tr = oracle.trace(view, splats, depth, eps, r_ov, first=first, mode=mode)
            sel = (tr.M > 0) if kind == "no M == b filter" else (tr.M == b)
            psi = oracle.shadow_dirs(tr, splats, [w], eps, mode)[0] * sel.astype(np.uint8)
            t = oracle.Trace(tr.M, tr.ids, tr.p, tr.n, tr.k, tr.u, tr.v, tr.path, psi)
            E = E + oracle.po_field(t, freqs_hz, w)[0]
        return E
    return fn


@pytest.fixture(scope="module")
def dihedral_geom():
    sc = scenes.dihedral(6000, seed=21)
    vd = scenes.aggregation_views(sc, 128, 128)
    S, gv, _, _ = oracle.build_geometry(sc, vd, "fp32")
    return sc, S, gv


@pytest.mark.parametrize("kind", ["receiver sign", "last bounce dropped",
                                  "full-depth trace at every b", "no M == b filter"])
def test_every_bounce_pin_catches_a_planted_mistake(kind, dihedral_geom, monkeypatch):
    monkeypatch.setattr(oracle, "po_field_every_bounce", _every_bounce_variant(kind))
    with pytest.raises(AssertionError):
        P.test_every_bounce_field_on_the_dihedral(dihedral_geom)


def test_every_bounce_variant_without_a_mistake_passes(dihedral_geom, monkeypatch):
    monkeypatch.setattr(oracle, "po_field_every_bounce", _every_bounce_variant("none"))
    P.test_every_bounce_field_on_the_dihedral(dihedral_geom)
