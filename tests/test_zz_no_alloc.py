"""The conservation record computed without allocating any memory
(lbm_conservation_noalloc), for callers that cannot call cudaMalloc: its
output must equal the handle-based lbm_conservation on the same state, on
two calls in a row (the second call reuses the fixed scratch the first one
left behind). Collected last on purpose; it also passes alone."""
import numpy as np
import pytest

from gpu_common import oracle_case, slab_fields

pytestmark = pytest.mark.gpu


# a periodic box, bounce-back walls (the pair force's density beyond a wall
# is the adjacent node's) with a body force and a hot segment, and an open
# bottom (the open state's density beyond it)
CASES = {"periodic": {}, "walls": dict(walls=1, accel_y=-1e-4, Tr_bottom=0.8, Tr_hot=0.95, hot_x0=90, hot_len=20),
         "open_bottom": dict(walls=1, open_sides=1, Tr_open=0.85)}


@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_record_matches_handle_record(gpu_lib, case):
    import torch
    from paper_2106_01557_gb300 import lbm

    nx, ny = 100, 37
    kw = CASES[case]
    o = oracle_case(nx, ny, **kw)
    fields = slab_fields(o, seed=31)
    cfg = lbm.default_config(nx, ny, precision="f64", **kw)
    h = lbm.Lattice(cfg)
    h.set_fields(*fields)
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    for call in range(2):
        h.step(7)
        ref = h.conservation()
        f, g = h.get_populations()
        fd = torch.from_numpy(f).cuda()
        gd = torch.from_numpy(g).cuda()
        torch.cuda.synchronize()
        lbm.conservation_noalloc(cfg, fd, gd, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got[0] == pytest.approx(ref[0], rel=1e-12), call
        scale = ref[0] * h.params()["c"]
        assert abs(got[1] - ref[1]) < 1e-12 * scale and abs(got[2] - ref[2]) < 1e-12 * scale
        assert got[3] == pytest.approx(ref[3], rel=1e-12)
        assert got[4] == pytest.approx(ref[4], rel=1e-12)
        assert got[5] == pytest.approx(ref[5], rel=1e-12)
        assert got[6] == 0.0


def test_noalloc_rejects_lattice_beyond_limit(gpu_lib):
    import torch
    from paper_2106_01557_gb300 import lbm

    cfg = lbm.default_config(2048, 1024, precision="f64")
    small = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.conservation_noalloc(cfg, small, small, small)
    assert e.value.code == -1 and "LBM_NOALLOC_MAX_NODES" in str(e.value)
