"""The allocation-free deposit (for callers that cannot call cudaMalloc) gives
the same density as the handle's deposit, bit for bit, on consecutive calls
that share its fixed scratch. Collected last on purpose."""
import numpy as np
import pytest

from paper_2312_02968_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_deposit_matches_handle_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2312_02968_gb300 import binding as B

    dev = torch.device("cuda", 0)
    cases = [(64, 1.5, W.isothermal(64, 1.0, 20000, 4.0, 25.0, seed=31)),
             (32, 1.0, W.uniform_random(32, 3000, seed=32))]
    for n, sigma, p in cases:  # two calls in a row, different size and width
        t = {k: torch.from_numpy(np.ascontiguousarray(p[k])).to(dev) for k in ("cell", "offset", "vel", "mass")}
        h = B.MondPM(n, 1, float(n), 1.0, 1.0, B.MU_DEEP, sigma, len(p["mass"]))
        h.bind_particles(t["cell"], t["offset"], t["vel"], t["mass"])
        h.deposit()
        want = h.get_field(B.FIELD_RHO)
        got = torch.full((n, n, n), float("nan"), dtype=torch.float32, device=dev)
        B.deposit_noalloc(n, 1.0, sigma, t["cell"], t["offset"], t["mass"], got)
        torch.cuda.synchronize()
        assert torch.equal(got.view(torch.int32), want.view(torch.int32))
        h.close()
    with pytest.raises(B.MondError):
        B.deposit_noalloc(256, 1.0, 1.0, t["cell"], t["offset"], t["mass"], got)
