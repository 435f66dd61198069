"""The unit-throughput probes (pe_probe_units) run, report the operation
counts their launch shapes imply, and give plausible orderings of the
rates; the full measurement is `python -m paper_2408_15583_gb300.peaks`."""
import math

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def test_operation_counts():
    from paper_2408_15583_gb300 import _lib
    lib = _lib.load()
    nbytes = 1 << 20
    buf = torch.zeros(nbytes, dtype=torch.uint8, device=DEV)
    s = torch.cuda.current_stream().cuda_stream
    blocks, it = 3, 5
    th = blocks * 256
    assert lib.pe_probe_units(0, blocks, it, buf.data_ptr(), nbytes, s) == th * it * 8 * 2
    assert lib.pe_probe_units(1, blocks, it, buf.data_ptr(), nbytes, s) == th * it * 8
    assert lib.pe_probe_units(2, blocks, it, buf.data_ptr(), nbytes, s) == th * it * 8 * 2
    assert lib.pe_probe_units(5, blocks, it, buf.data_ptr(), nbytes, s) == th * it * 8 * 4
    buf.zero_()
    assert lib.pe_probe_units(3, blocks, it, buf.data_ptr(), nbytes, s) == (nbytes - 16) * it
    buf.fill_(255)
    assert lib.pe_probe_units(4, blocks, it, buf.data_ptr(), nbytes, s) == th * it
    torch.cuda.synchronize()
    # the atomics lowered some of the all-ones keys, and only inside the table
    w = buf.view(torch.int64)
    assert int((w != -1).sum()) > 0


def test_short_measurement_is_plausible():
    from paper_2408_15583_gb300 import peaks
    r = peaks.measure(DEV, reps=1, scale=0.05)
    for name in peaks.PROBES:
        v = r[name]["value"]
        assert math.isfinite(v) and v > 0, name
    # FP32 FMA outruns FP64 FMA and the sine path on this part
    assert r["fp32_fma"]["value"] > r["fp64_fma"]["value"]
    assert r["fp32_fma"]["value"] * 1e12 / 2 > r["sin"]["value"] * 1e9
