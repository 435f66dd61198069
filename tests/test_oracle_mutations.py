"""The oracle's pins must catch plausible mistakes in the steps they cover.

One mistake at a time is planted in a copy of the oracle's C source (a
textual replacement that must match exactly once, so this test breaks loudly
when the source moves), the copy is built into its own library with the
oracle's own compiler flags, and the pins covering that step run against it:
at least one must fail.  The planted mistakes change arithmetic only (signs,
comparisons, dropped terms, constants), never an index or a size, so no
mutant can read or write out of bounds.  The every-bounce composition and
the Python steps are mutated by replacing the function; the FP64 reference
network (oracle/unet.py) by executing its source with one textual change.
CPU only.
"""
import os
import shutil

import numpy as np
import pytest

import oracle
import scenes
import test_oracle_grid as G
import test_oracle_pins as P
import test_unet_oracle as U
from oracle import unet

# name, file, original text, planted text, pins (callables taking the
# dihedral geometry built by the unchanged oracle; most ignore it)
C_MUTANTS = [
    # PO (Eq. 5-14)
    ("PO: sinc over v' dropped", "oracle.c",
     "double amp = area * sinc(0.5 * dot3(q, up)) * sinc(0.5 * dot3(q, vp));",
     "double amp = area * sinc(0.5 * dot3(q, up));",
     [lambda g: P.test_po_parallelogram_cells_use_cross_product_area(),
      lambda g: P.test_bistatic_plate_exact_integral_and_receiver_shadowing(40.0)]),
    ("PO: cell area as |u'| |v'| instead of |u' x v'|", "oracle.c",
     "double area = sqrt(dot3(cr, cr));",
     "double area = sqrt(dot3(up, up)) * sqrt(dot3(vp, vp));",
     [lambda g: P.test_po_parallelogram_cells_use_cross_product_area()]),
    ("PO: phase sign", "oracle.c",
     "double cre = cos(ph), cim = -sin(ph);",
     "double cre = cos(ph), cim = sin(ph);",
     [lambda g: P.test_po_translation_phase_convention()]),
    ("PO: V-polarisation sign", "oracle.c",
     "h[0][c] = -vl[c] / lv;",
     "h[0][c] = vl[c] / lv;",
     [lambda g: P.test_bistatic_plate_exact_integral_and_receiver_shadowing(15.0)]),
    ("PO: u' and v' projections swapped", "oracle.c",
     "nu = dot3(nl, ul) / nk, nv = dot3(nl, vl) / nk;",
     "nu = dot3(nl, vl) / nk, nv = dot3(nl, ul) / nk;",
     [lambda g: P.test_po_parallelogram_cells_use_cross_product_area(),
      lambda g: P.test_po_plate_pattern_textbook(25.0)]),
    ("PO: sign of k_s in q", "oracle.c",
     "q[c] = kw * (kl[c] - ks[c]);",
     "q[c] = kw * (kl[c] + ks[c]);",
     [lambda g: P.test_po_plate_pattern_textbook(25.0)]),
    # Alg. 1 and the finite heap
    ("pixel rays through pixel corners, not centres", "oracle_core.h",
     "R fi = ((R)i + (R)0.5) - (R)0.5 * (R)v->W;",
     "R fi = (R)i - (R)0.5 * (R)v->W;",
     [lambda g: P.test_gfb_single_disk_handmade("fp32")]),
    ("Alg. 1 tube: score along the ray instead of Length(p - o)", "oracle_core.h",
     "*score = SQRT(SFX(dot)(q, q));",
     "*score = t;",
     [lambda g: P.test_gfb_tube_mode_handmade("fp32")]),
    ("Alg. 1 tube: candidates behind the screen kept", "oracle_core.h",
     "if (!(t > (R)0)) return 0;\n  *score",
     "if (0) return 0;\n  *score",
     [lambda g: P.test_gfb_tube_mode_handmade("fp32"),
      lambda g: P.test_alg1_large_k_equals_the_unbounded_heap()]),
    ("Alg. 1: ties to the larger index", "oracle_core.h",
     "if (t < *best || (t == *best && s < *bi)) {",
     "if (t < *best || (t == *best && s > *bi)) {",
     [lambda g: P.test_gfb_nearest_and_tie_break("fp32")]),
    ("finite K: the farthest kept candidate", "oracle_core.h",
     "if (ks[e] < best || (ks[e] == best && ki[e] < bi)) {",
     "if (ks[e] > best || best == (R)INFINITY || (ks[e] == best && ki[e] < bi)) {",
     [lambda g: P.test_alg1_finite_k_hand_case("fp32")]),
    ("finite K: heap kept in the wrong order", "oracle_core.h",
     "while (at > 0 && ka[at - 1] > a) {",
     "while (at > 0 && ka[at - 1] < a) {",
     [lambda g: P.test_alg1_finite_k_hand_case("fp32")]),
    # Alg. 3, aggregation steps: edge rule, Canny, fusion, Eq. 22
    ("edge rule dropped", "oracle_core.h",
     "if (dt > tauL) return 1;",
     "if (dt > tauL && 0) return 1;",
     [lambda g: P.test_edge_filter_handmade()]),
    ("Canny: no hysteresis (low threshold = high)", "oracle_core.h",
     "const R high = ((R)8 * tau) * L, low = (R)0.5 * high;",
     "const R high = ((R)8 * tau) * L, low = high;",
     [lambda g: P.test_canny_weak_step_alone_and_joined_to_a_strong_one("fp32")]),
    ("Canny: high threshold halved", "oracle_core.h",
     "const R high = ((R)8 * tau) * L, low = (R)0.5 * high;",
     "const R high = ((R)4 * tau) * L, low = (R)0.5 * high;",
     [lambda g: P.test_canny_ramp_threshold_and_flat_map("fp32"),
      lambda g: P.test_canny_weak_step_alone_and_joined_to_a_strong_one("fp32")]),
    ("fusion: normals not turned into one hemisphere", "oracle_core.h",
     "if (SFX(dot)(nn, E0->n) < (R)0)",
     "if (SFX(dot)(nn, E0->n) < (R)0 && 0)",
     [lambda g: P.test_fusion_average_over_views("fp32")]),
    ("fusion: radius of the first contributor, not the largest", "oracle_core.h",
     "if (r > rmax) rmax = r;",
     "if (rmax == 0.0) rmax = r;",
     [lambda g: P.test_fusion_owner_is_the_most_frontal_view("fp32")]),
    ("fusion: centre divided by count + 1", "oracle_core.h",
     "S->c[k] = (R)(sp3[k] / cnt);",
     "S->c[k] = (R)(sp3[k] / (cnt + 1.0));",
     [lambda g: P.test_fusion_average_over_views("fp32")]),
    ("fusion: owner ties go to the later view", "oracle_core.h",
     "if (sc > best) {",
     "if (sc >= best) {",
     [lambda g: P.test_fusion_owner_is_the_most_frontal_view("fp32")]),
    ("Eq. 22: sqrt(2) replaced by 1.5", "oracle_core.h",
     "if (s < 2.5) return (1.4142135623730951 * L) * s;",
     "if (s < 2.5) return (1.5 * L) * s;",
     [lambda g: P.test_eq22_radius_values("fp64")]),
    # Alg. 3, bounce loop: bounces, Eq. 23, epsilon, Psi
    ("Eq. 4: reflection sign", "oracle_core.h",
     "for (int k = 0; k < 3; ++k) out[k] = a[k] - s * n[k];",
     "for (int k = 0; k < 3; ++k) out[k] = a[k] + s * n[k];",
     [lambda g: P.test_trihedral_axis_triple_bounce_aperture()]),
    ("tube vector u not reflected", "oracle_core.h",
     "SFX(reflect)(u, nn, ru);",
     "for (int k = 0; k < 3; ++k) ru[k] = u[k];",
     [lambda g: P.test_trihedral_axis_triple_bounce_aperture(),
      lambda g: P.test_rcs_dihedral_realised_aperture(g),
      lambda g: P.test_rolled_dihedral_twist_and_reciprocity()]),
    ("tube vector v not reflected", "oracle_core.h",
     "SFX(reflect)(v, nn, rv);",
     "for (int k = 0; k < 3; ++k) rv[k] = v[k];",
     [lambda g: P.test_rolled_dihedral_twist_and_reciprocity()]),
    ("path: later segments counted half", "oracle_core.h",
     "path = path + sqrt((dx * dx + dy * dy) + dz * dz);",
     "path = path + 0.5 * sqrt((dx * dx + dy * dy) + dz * dz);",
     [lambda g: P.test_epsilon_minimum_travel("fp32"),
      lambda g: P.test_rcs_dihedral_realised_aperture(g)]),
    ("Psi: shadow ray toward the transmitter's back", "oracle_core.h",
     "R w[3] = {-V.d[0], -V.d[1], -V.d[2]};",
     "R w[3] = {V.d[0], V.d[1], V.d[2]};",
     [lambda g: P.test_bistatic_psi_toward_the_transmitter_is_the_monostatic_psi(),
      lambda g: P.test_dihedral_interior_rays_bounce_twice(g)]),
    ("bistatic Psi: shadow rays start at t > 0 instead of t > eps", "oracle_core.h",
     "const R E = (R)eps;\n  for (int o = 0; o < nobs; ++o) {",
     "const R E = (R)0;\n  for (int o = 0; o < nobs; ++o) {",
     [lambda g: P.test_bistatic_psi_toward_the_transmitter_is_the_monostatic_psi()]),
    ("bistatic Psi: blocked and visible swapped", "oracle_core.h",
     "psi = SFX(any_hit)(&S, pq, w, E) ? 0 : 1;",
     "psi = SFX(any_hit)(&S, pq, w, E) ? 1 : 0;",
     [lambda g: P.test_bistatic_plate_exact_integral_and_receiver_shadowing(15.0),
      lambda g: P.test_bistatic_psi_toward_the_transmitter_is_the_monostatic_psi()]),
    ("Eq. 23: no overlap window", "oracle_core.h",
     "R lim = tb + r_ov;",
     "R lim = tb;",
     [lambda g: P.test_eq23_overlap_select_and_blend("fp32")]),
    ("nearest hit replaced by the farthest", "oracle_core.h",
     "if (t < *tb || (t == *tb && s < *sb)) {",
     "if (*tb == (R)INFINITY || t > *tb) {",
     [lambda g: P.test_eq23_overlap_select_and_blend("fp32"),
      lambda g: P.test_epsilon_minimum_travel("fp32")]),
    ("Eq. 23: blend weight rho instead of 1 - rho", "oracle_core.h",
     "R w = (R)1 - rho;",
     "R w = rho;",
     [lambda g: P.test_eq23_overlap_select_and_blend("fp32")]),
    ("epsilon ignored on bounces", "oracle_core.h",
     "R E = (R)eps, RO = (R)r_ov;",
     "R E = (R)0, RO = (R)r_ov;",
     [lambda g: P.test_epsilon_minimum_travel("fp32")]),
    # the field's compensated sum (Neumaier)
    ("Neumaier: correction of the first branch with its sign flipped", "oracle.c",
     "a->c += (a->s - t) + x;",
     "a->c += (t - a->s) + x;",
     [lambda g: P.test_neumaier_sum_against_exact_rational_sums()]),
    ("Neumaier: no branch for a term larger than the sum (Kahan's form)", "oracle.c",
     "if (fabs(a->s) >= fabs(x))",
     "if (1)",
     [lambda g: P.test_neumaier_sum_against_exact_rational_sums()]),
    ("Neumaier: the two branches swapped", "oracle.c",
     "if (fabs(a->s) >= fabs(x))",
     "if (fabs(a->s) < fabs(x))",
     [lambda g: P.test_neumaier_sum_against_exact_rational_sums()]),
    ("field: the compensation term dropped", "oracle.c",
     "acc[pol][c][ri].s + acc[pol][c][ri].c;",
     "acc[pol][c][ri].s;",
     [lambda g: P.test_po_field_keeps_a_term_below_the_running_sums_ulp()]),
    # the uniform grid of the large searches (must equal brute force)
    ("grid: elements listed only in their centre's cell", "oracle_grid.h",
     "double ri = fabs(r[i]) + pad;",
     "double ri = pad;",
     [lambda g: G.grid_equals_brute("dihedral"), lambda g: G.grid_equals_brute("octar")]),
    ("grid: first boundary of a backward walk one cell off", "oracle_grid.h",
     "w->tmax[k] = (g->lo[k] + i * g->cell - o[k]) / d[k];",
     "w->tmax[k] = (g->lo[k] + (i - 1) * g->cell - o[k]) / d[k];",
     [lambda g: G.grid_equals_brute("dihedral"), lambda g: G.grid_equals_brute("octar")]),
    ("grid: walk stops a cell before the bound", "oracle_grid.h",
     "if (!w->live || w->t_in > t_stop + w->g->slack) return 0;",
     "if (!w->live || w->t_in > t_stop - w->g->cell) return 0;",
     [lambda g: G.grid_equals_brute("dihedral"), lambda g: G.grid_equals_brute("octar")]),
    ("grid: Eq. 23 candidates in walk order, with repeats", "oracle_grid.h",
     "  if (L->n < 2) return;",
     "  return;",
     [lambda g: G.grid_equals_brute("dihedral"), lambda g: G.grid_equals_brute("octar")]),
    ("grid: Eq. 23 candidates only up to the nearest hit", "oracle_core.h",
     "SFX(candidates)(S, o, d, tmin, lim, &L);",
     "SFX(candidates)(S, o, d, tmin, tb, &L);",
     [lambda g: G.grid_equals_brute("dihedral"), lambda g: G.grid_equals_brute("octar"),
      lambda g: G.grid_equals_brute("composite")]),
    # surfel attributes
    ("k-NN: squared distance without its z term", "oracle.c",
     "float d2 = (dx * dx + dy * dy) + dz * dz;",
     "float d2 = (dx * dx + dy * dy) + 0.0f * dz;",
     [lambda g: P.test_knn_distances_match_an_independent_kd_tree()]),
]


@pytest.fixture
def plant(tmp_path):
    """plant(file, old, new): build a copy of the oracle with one textual
    change and make it the oracle's library until the test ends."""
    src = os.path.dirname(oracle.__file__)
    saved = oracle._lib

    def _plant(fname, old, new):
        for f in ("oracle.c", "oracle_core.h", "oracle_grid.h"):
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


def _failing(pins, geom):
    caught = []
    for pin in pins:
        try:
            pin(geom)
        except AssertionError:
            caught.append(pin)
    return caught


def test_an_unchanged_copy_passes_the_pins(plant, dihedral_geom):
    # the mechanism itself (copy, flags, binding) changes nothing
    name, fname, old, _, _ = C_MUTANTS[0]
    plant(fname, old, old)
    pins = [p for m in C_MUTANTS for p in m[4]]
    assert _failing(pins, dihedral_geom) == []


@pytest.mark.parametrize("mutant", C_MUTANTS, ids=[m[0] for m in C_MUTANTS])
def test_pins_catch_a_planted_mistake(mutant, plant, dihedral_geom):
    name, fname, old, new, pins = mutant
    plant(fname, old, new)
    assert _failing(pins, dihedral_geom), f"no pin caught: {name}"


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


# ----------------------------------------------------------------------------
# steps written in Python: sigma, the k-NN radius, the normal's orientation
# ----------------------------------------------------------------------------

def _sigma_quarter(real):
    return lambda E, freqs_hz, u_hat, v_hat: 0.25 * real(E, freqs_hz, u_hat, v_hat)


def _radius_over_k_plus_one(real):
    def fn(idx, d2, self_idx, k_r):
        return (real(idx, d2, self_idx, k_r).astype(np.float64) * k_r / (k_r + 1)).astype(np.float32)
    return fn


def _normals_flipped(real):
    def fn(pos, k_r=8, k_n=16, ref=None):
        r, n, w, rest = real(pos, k_r, k_n, ref=ref)
        return r, -n, w, rest
    return fn


PY_MUTANTS = [
    ("sigma: k^2 / (4 pi) instead of k^2 / pi", "sigma_from_field", _sigma_quarter,
     [P.test_rcs_sphere_surfels_vs_exact_po]),
    ("k-NN radius: mean over k_r + 1", "knn_radius", _radius_over_k_plus_one,
     [P.test_knn_radius_and_normal_on_a_square_lattice]),
    ("PCA normal: orientation flipped", "point_attributes", _normals_flipped,
     [P.test_knn_radius_and_normal_on_a_square_lattice,
      P.test_pca_normal_of_a_tilted_plane_and_duplicates]),
]


@pytest.mark.parametrize("mutant", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_python_steps_catch_a_planted_mistake(mutant, monkeypatch):
    name, attr, make, pins = mutant
    monkeypatch.setattr(oracle, attr, make(getattr(oracle, attr)))
    caught = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            caught += 1
    assert caught, f"no pin caught: {name}"


# ----------------------------------------------------------------------------
# the FP64 reference network and its losses (oracle/unet.py)
# ----------------------------------------------------------------------------

UNET_MUTANTS = [
    ("depth head added to nothing (no residual on the coarse depth)",
     'out["depth"] = out["depth"] + x', 'out["depth"] = out["depth"]',
     [U.test_depth_output_refines_the_input]),
    ("ConvNeXt residual dropped", "    return x + y\n", "    return y\n",
     [U.test_convnext_block_is_identity_with_zero_last_projection,
      U.test_convnext_block_closed_form_gelu]),
    ("ReLU instead of GELU", "y = F.gelu(conv1(", "y = F.relu(conv1(",
     [U.test_convnext_block_closed_form_gelu]),
    ("Eq. 19: alpha and 1 - alpha swapped",
     "foc = torch.where(hit, -alpha * (1 - p) ** gamma * logp, -(1 - alpha) * p ** gamma * log1mp)",
     "foc = torch.where(hit, -(1 - alpha) * (1 - p) ** gamma * logp, -alpha * p ** gamma * log1mp)",
     [U.test_focal_loss_closed_values]),
    ("Eq. 19: gamma - 1", "-alpha * (1 - p) ** gamma * logp", "-alpha * (1 - p) ** (gamma - 1) * logp",
     [U.test_focal_loss_closed_values]),
    ("Eq. 21: factors of L2 and L3 swapped",
     "L = 1.0 * L1 + 0.5 * L2 + 1.0 * L3 + 0.5 * L4",
     "L = 1.0 * L1 + 1.0 * L2 + 0.5 * L3 + 0.5 * L4",
     [U.test_normal_depth_and_gradient_losses_closed_values]),
    ("Eq. 17: absolute instead of squared difference",
     "L1 = ((d - d_gt) ** 2)[hit].sum() / nh", "L1 = (d - d_gt).abs()[hit].sum() / nh",
     [U.test_normal_depth_and_gradient_losses_closed_values]),
    ("Eq. 18: no division by |n| |n_gt|",
     "cn = _cross_norm(n, n_gt) / (torch.linalg.norm(n, dim=-1) * torch.linalg.norm(n_gt, dim=-1) + DIV_EPS)",
     "cn = _cross_norm(n, n_gt)",
     [U.test_normal_depth_and_gradient_losses_closed_values]),
    ("Eq. 20: central difference without the 1/2",
     "gu = 0.5 * (dd[:, 1:-1, 2:] - dd[:, 1:-1, :-2])", "gu = (dd[:, 1:-1, 2:] - dd[:, 1:-1, :-2])",
     [U.test_normal_depth_and_gradient_losses_closed_values]),
]


def _unet_variant(old, new, monkeypatch):
    """Execute oracle/unet.py with one textual change and route the module's
    entry points to the changed code."""
    with open(unet.__file__) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation site not found exactly once: {old!r}"
    ns = {"__name__": "unet_variant"}
    exec(compile(src.replace(old, new), unet.__file__ + " (variant)", "exec"), ns)
    for attr in ("forward", "losses", "convnext"):
        monkeypatch.setattr(unet, attr, ns[attr])


def _caught(pins):
    n = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            n += 1
    return n


def test_unet_unchanged_variant_passes_the_pins(monkeypatch):
    _unet_variant("    return x + y\n", "    return x + y\n", monkeypatch)
    assert _caught([p for m in UNET_MUTANTS for p in m[3]]) == 0


@pytest.mark.parametrize("mutant", UNET_MUTANTS, ids=[m[0] for m in UNET_MUTANTS])
def test_unet_pins_catch_a_planted_mistake(mutant, monkeypatch):
    name, old, new, pins = mutant
    _unet_variant(old, new, monkeypatch)
    assert _caught(pins), f"no pin caught: {name}"


# ----------------------------------------------------------------------------
# the view frame (oracle/__init__.py, Python)
# ----------------------------------------------------------------------------

VIEW_MUTANTS = [
    ("u = -theta_hat", "u = [ct * cp, ct * sp, -st]", "u = [-ct * cp, -ct * sp, st]"),
    ("screen one pitch too close", "D = float(extent) + L", "D = float(extent)"),
    ("phi measured the other way", "w = [st * cp, st * sp, ct]", "w = [st * cp, -st * sp, ct]"),
]


@pytest.mark.parametrize("mutant", VIEW_MUTANTS, ids=[m[0] for m in VIEW_MUTANTS])
def test_view_frame_pin_catches_a_planted_mistake(mutant, monkeypatch):
    name, old, new = mutant
    with open(oracle.__file__) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation site not found exactly once: {old!r}"
    # under the oracle's own module name: dataclasses look their module up
    ns = {"__name__": oracle.__name__, "__file__": oracle.__file__}
    exec(compile(src.replace(old, new), oracle.__file__ + " (variant)", "exec"), ns)
    monkeypatch.setattr(oracle, "view_from_angles", ns["view_from_angles"])
    caught = 0
    for mode in ("fp32", "fp64"):
        try:
            P.test_view_frame_is_the_spherical_basis(mode)
        except AssertionError:
            caught += 1
    assert caught == 2, f"not caught in both modes: {name}"
