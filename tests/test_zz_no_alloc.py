"""The allocation-free deposit, for callers that cannot call cudaMalloc (a host
framework that owns every device allocation, a plug-in that must not grow the
process's device footprint). It must give the same density as the handle's
deposit and as the CPU oracle, bit for bit, on consecutive calls that share its
fixed scratch, at the edges of that scratch (128^3 cells, kernel width 2 px,
the smallest 8^3 domain), when a call returns to an earlier kernel width (the
table is rebuilt), and after the device was reset between two calls (the
scratch is set up again). Collected last on purpose."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_2312_02968_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def _oracle_rho(n, s, sigma, p):
    acc, ka, _ = oracle.deposit_fixed(n, sigma, p["cell"], p["offset"], p["mass"])
    r32, _ = oracle.acc_to_rho(acc, ka, s)
    return r32


def _noalloc(B, n, s, sigma, t, dev):
    got = torch.full((n, n, n), float("nan"), dtype=torch.float32, device=dev)
    B.deposit_noalloc(n, s, sigma, t["cell"], t["offset"], t["mass"], got)
    torch.cuda.synchronize()
    return got


def test_noalloc_deposit_matches_handle_twice():
    _need_gpu()
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
        got = _noalloc(B, n, 1.0, sigma, t, dev)
        assert torch.equal(got.view(torch.int32), want.view(torch.int32))
        h.close()
    got = torch.empty((8, 8, 8), dtype=torch.float32, device=dev)
    with pytest.raises(B.MondError):
        B.deposit_noalloc(256, 1.0, 1.0, t["cell"], t["offset"], t["mass"], got)
    with pytest.raises(B.MondError):
        B.deposit_noalloc(32, 1.0, 2.5, t["cell"], t["offset"], t["mass"], got)


def test_noalloc_deposit_at_its_limits_matches_oracle():
    """128^3 cells and kernel width 2 px (the 2103-tap ball, 15-word table
    rows) with 1e5 clustered particles; the 8^3 domain at width 0.75 px, where
    every ball wraps the periodic faces; then width 2 again on 128^3 (the table
    rebuilt from the value an earlier call left). Each density equals the
    oracle's fixed-point deposit bit for bit."""
    _need_gpu()
    from paper_2312_02968_gb300 import binding as B

    dev = torch.device("cuda", 0)
    big = W.isothermal(128, 1.0, 100_000, 4.0, 51.2, seed=41)
    tiny = W.uniform_random(8, 500, seed=42)
    mid = W.isothermal(64, 0.5, 30_000, 3.0, 25.0, seed=43)
    for n, s, sigma, p in ((128, 1.0, 2.0, big), (8, 1.0, 0.75, tiny), (64, 0.5, 1.5, mid), (128, 1.0, 2.0, big)):
        t = {k: torch.from_numpy(np.ascontiguousarray(p[k])).to(dev) for k in ("cell", "offset", "mass")}
        got = _noalloc(B, n, s, sigma, t, dev).cpu().numpy()
        want = _oracle_rho(n, s, sigma, p)
        assert np.array_equal(got.view(np.int32), want.view(np.int32)), (n, sigma)


_CHILD = r"""
import ctypes, os, sys
import numpy as np
sys.path.insert(0, os.environ["MOND_ROOT"])
from paper_2312_02968_gb300 import binding as B
rt = None
for name in ("libcudart.so", "libcudart.so.13", "libcudart.so.12"):
    try:
        rt = ctypes.CDLL(name)
        break
    except OSError:
        pass
if rt is None:
    import torch  # only to locate the runtime library it ships with
    d = os.path.join(os.path.dirname(torch.__file__), "lib")
    cands = [f for f in os.listdir(d) if f.startswith("libcudart")]
    rt = ctypes.CDLL(os.path.join(d, cands[0]))
L = B.lib()
data = np.load(sys.argv[1])
n, s, sigma = int(data["n"]), float(data["s"]), float(data["sigma"])
outs = []
for rep in range(2):
    ptrs = []
    for k in ("cell", "offset", "mass"):
        a = np.ascontiguousarray(data[k])
        p = ctypes.c_void_p()
        assert rt.cudaMalloc(ctypes.byref(p), ctypes.c_size_t(a.nbytes)) == 0
        assert rt.cudaMemcpy(p, a.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(a.nbytes), 1) == 0
        ptrs.append(p)
    out = ctypes.c_void_p()
    assert rt.cudaMalloc(ctypes.byref(out), ctypes.c_size_t(4 * n ** 3)) == 0
    rc = L.mond_pm_deposit_noalloc(n, ctypes.c_double(s), ctypes.c_double(sigma), ctypes.c_int64(len(data["mass"])),
                                   ptrs[0], ptrs[1], ptrs[2], out, None)
    assert rc == 0, L.mond_pm_last_error(None)
    assert rt.cudaDeviceSynchronize() == 0
    h = np.empty((n, n, n), np.float32)
    assert rt.cudaMemcpy(h.ctypes.data_as(ctypes.c_void_p), out, ctypes.c_size_t(h.nbytes), 2) == 0
    outs.append(h)
    # ends this process's own context: the module and its __device__ scratch go with it
    assert rt.cudaDeviceReset() == 0
np.save(sys.argv[2], np.stack(outs))
"""


def test_noalloc_deposit_after_device_reset(tmp_path):
    """A fresh process calls the entry point, resets its device (which ends
    only its own context), and calls again with the same kernel width: the
    second call must set its scratch up in the new context and give the same
    density, equal to the oracle's."""
    _need_gpu()
    p = W.isothermal(32, 1.0, 5000, 2.0, 12.0, seed=44)
    inp = tmp_path / "in.npz"
    out = tmp_path / "out.npy"
    np.savez(inp, n=32, s=1.0, sigma=1.5, cell=p["cell"], offset=p["offset"], mass=p["mass"])
    env = dict(os.environ, MOND_ROOT=ROOT)
    r = subprocess.run([sys.executable, "-c", _CHILD, str(inp), str(out)], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    got = np.load(out)
    want = _oracle_rho(32, 1.0, 1.5, p)
    for k in range(2):
        assert np.array_equal(got[k].view(np.int32), want.view(np.int32)), k
