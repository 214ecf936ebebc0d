"""ctypes binding of the C ABI in include/mond_pm.h.

Argument marshalling only: every step of the method runs in the CUDA library
``_build/libmondpm.so``. PyTorch provides device memory (the workspace and the
particle tensors) and the CUDA stream. ``lib()`` raises if the library has not
been built; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmondpm.so")

MU_DEEP, MU_SIMPLE, MU_STANDARD, MU_NEWTON = 0, 1, 2, 3
WARM_NONE, WARM_PREV, WARM_GUESS, WARM_GUESS_RAW, WARM_INCREMENT = 0, 1, 2, 3, 4
FIELD_RHO, FIELD_GN, FIELD_H, FIELD_PHI, FIELD_ACC, FIELD_SMOOTH, FIELD_GM = 0, 1, 2, 3, 4, 5, 6
DENS_BARYONIC, DENS_APPARENT, DENS_PHANTOM = 0, 1, 2
OPT_KEEP_PHI, OPT_TRACK_DH, OPT_USE_GRAPH, OPT_TIMING, OPT_PIPELINED, OPT_CHUNK, OPT_GATHER = 1, 2, 3, 4, 5, 6, 7
OPT_TEST_LOST_LOAD = 8  # tests of the bounded device waits only
OPT_CYCLE_MEAN = 9
OPT_FOLD = 10
OPT_GRID_CAP = 11
ERRORS = {0: "MOND_OK", -1: "MOND_EINVAL", -2: "MOND_ENOMEM", -3: "MOND_ECUDA", -4: "MOND_EOVERFLOW",
          -5: "MOND_EDOMAIN", -6: "MOND_ENAN", -7: "MOND_ETIMEOUT", -8: "MOND_ESTATE"}

# every function the header declares, with (restype, argtypes)
_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double


class Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("pad", ctypes.c_int32)]


class Diag(ctypes.Structure):
    _fields_ = [("mass", _D), ("momentum", _D * 3), ("com", _D * 3), ("ang_mom", _D * 3), ("e_kin", _D),
                ("e_pot", _D), ("rho_mass", _D), ("n_iter_done", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("dH", _D * 64)]


class KStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", _I64), ("ms", _D), ("bytes", _D)]


SIGNATURES = {
    "mond_pm_workspace_bytes": (_I, [Grid, _D, _I64, ctypes.POINTER(ctypes.c_size_t)]),
    "mond_pm_create": (_I, [Grid, _D, _D, _D, _I, _D, _P, _P, ctypes.c_size_t, _I64, ctypes.POINTER(_P)]),
    "mond_pm_destroy": (_I, [_P]),
    "mond_pm_set_option": (_I, [_P, _I, _I64]),
    "mond_pm_bind_particles": (_I, [_P, _I64, _P, _P, _P, _P]),
    "mond_pm_deposit": (_I, [_P]),
    "mond_pm_set_density": (_I, [_P, _P]),
    "mond_pm_solve_field": (_I, [_P, _I, _I, _P]),
    "mond_pm_smooth": (_I, [_P, _P]),
    "mond_pm_gather_push": (_I, [_P, _D]),
    "mond_pm_half_kick": (_I, [_P, _D]),
    "mond_pm_gather": (_I, [_P, _P]),
    "mond_pm_density": (_I, [_P, _I, _P]),
    "mond_pm_set_dipole_layer": (_I, [_P, _I, _D]),
    "mond_pm_set_h_state": (_I, [_P, _P]),
    "mond_pm_increment_workspace_bytes": (_I, [Grid, ctypes.POINTER(ctypes.c_size_t)]),
    "mond_pm_set_increment_workspace": (_I, [_P, _P, ctypes.c_size_t]),
    "mond_pm_shell_mass": (_I, [_P, _I, ctypes.POINTER(_D), _D, _I, ctypes.POINTER(_D)]),
    "mond_pm_box_mass": (_I, [_P, _I, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                              ctypes.POINTER(_D)]),
    "mond_pm_step": (_I, [_P, _D, _I, _I]),
    "mond_pm_step_host": (_I, [_P, _D, _I, _I, _P, _P, _P]),
    "mond_pm_diagnostics": (_I, [_P, ctypes.POINTER(Diag)]),
    "mond_pm_get_field": (_I, [_P, _I, _P]),
    "mond_pm_field_ptr": (_I, [_P, _I, ctypes.POINTER(_P)]),
    "mond_pm_get_deposit_acc": (_I, [_P, _P, ctypes.POINTER(ctypes.c_int32)]),
    "mond_pm_sync": (_I, [_P]),
    "mond_pm_last_error": (ctypes.c_char_p, [_P]),
    "mond_pm_kernel_launches": (_I64, [_P]),
    "mond_pm_kernel_stats": (_I, [_P, ctypes.POINTER(KStat), _I, ctypes.POINTER(_I)]),
    "mond_pm_deposit_noalloc": (_I, [ctypes.c_int32, _D, _D, _I64, _P, _P, _P, _P, _P]),
    "mond_pm_probe_smem_atomics": (_I, [_I, _P, ctypes.POINTER(_D)]),
    "mond_pm_batch_create": (_I, [_I, ctypes.POINTER(_P), _P, ctypes.POINTER(_P)]),
    "mond_pm_batch_step": (_I, [_P, _D, _I, _I, _I]),
    "mond_pm_batch_sync": (_I, [_P]),
    "mond_pm_batch_kernel_launches": (_I64, [_P]),
    "mond_pm_batch_destroy": (_I, [_P]),
    "mond_pm_autotune": (_I, [_P, _I, _I, ctypes.POINTER(_I64), ctypes.POINTER(_I)]),
}


class FnoShape(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("width", ctypes.c_int32), ("modes", ctypes.c_int32),
                ("layers", ctypes.c_int32)]


_F = ctypes.c_float
SIGNATURES.update({
    "mond_fno_param_count": (_I, [FnoShape, ctypes.POINTER(_I64)]),
    "mond_fno_workspace_bytes": (_I, [FnoShape, ctypes.POINTER(ctypes.c_size_t)]),
    "mond_fno_init": (_I, [FnoShape, ctypes.c_uint64, _P, _P]),
    "mond_fno_cast": (_I, [FnoShape, _P, _P, _P]),
    "mond_fno_forward": (_I, [FnoShape, _P, _P, _P, _P, _P]),
    "mond_fno_backward": (_I, [FnoShape, _P, _P, _P, _P, _P, _P]),
    "mond_fno_loss": (_I, [_I64, _P, _P, _P, _F, _P, _P]),
    "mond_fno_adam": (_I, [_I64, _P, _P, _P, _P, _F, _F, _F, _F, _I, _F, _P, _P]),
    "mond_fno_input": (_I, [_I, _I, _F, _P, _P, _P, _P]),
    "mond_fno_output": (_I, [_I, _I, _P, _P, _P, _P, _P]),
    "mond_fno_output_scratch_bytes": (ctypes.c_size_t, [_I, _I]),
    "mond_fno_coarsen": (_I, [_I, _I, _I, _P, _P, _P, _P, _P]),
    "mond_fno_mixture_density": (_I, [_I, _D, _I, _P, _P, _P, _P, _F, _P, _P]),
})

_lib = None


def lib():
    """Load libmondpm.so (raises if it was not built: run __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class MondError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def workspace_bytes(n: int, pad: int, kernel_width: float, max_particles: int) -> int:
    out = ctypes.c_size_t(0)
    rc = lib().mond_pm_workspace_bytes(Grid(n, pad), float(kernel_width), int(max_particles), ctypes.byref(out))
    if rc != 0:
        raise MondError(rc, "unsupported grid or kernel width")
    return int(out.value)


def deposit_noalloc(n_f: int, s: float, kernel_width: float, cell, offset, mass, rho_out, stream=None):
    """Density of the particles on an n_f^3 domain into rho_out (device
    float32 [n_f, n_f, n_f]) without allocating device memory: the library
    keeps fixed-size scratch for this call (n_f <= 128). For callers that
    cannot call cudaMalloc. Uses torch's current stream unless one is given."""
    import torch

    st = stream if stream is not None else torch.cuda.current_stream()
    rc = lib().mond_pm_deposit_noalloc(int(n_f), float(s), float(kernel_width), int(mass.numel()), _ptr(cell),
                                       _ptr(offset), _ptr(mass), _ptr(rho_out), ctypes.c_void_p(st.cuda_stream))
    if rc != 0:
        raise MondError(rc, lib().mond_pm_last_error(None).decode())


def probe_smem_atomics(bits: int = 32, stream=None) -> float:
    """Measured no-return shared-memory atomic adds per second on the current
    device (the deposit's roofline peak); a measurement, not the method."""
    import torch

    st = stream if stream is not None else torch.cuda.current_stream()
    out = ctypes.c_double()
    rc = lib().mond_pm_probe_smem_atomics(int(bits), ctypes.c_void_p(st.cuda_stream), ctypes.byref(out))
    if rc != 0:
        raise MondError(rc, "shared-memory atomic probe failed")
    return out.value


class MondPM:
    """One simulation handle: mesh n^3 (FFT domain (n pad)^3), box side, a0, G,
    interpolation function, Gaussian width in pixels. Workspace is a torch
    uint8 tensor on the current CUDA device; the handle runs on ``stream``
    (default: torch's current stream)."""

    def __init__(self, n: int, pad: int, box: float, a0: float, G: float, mu_kind: int, kernel_width: float,
                 max_particles: int, stream=None, device=None):
        import torch

        self.torch = torch
        self.n, self.pad, self.nf = n, pad, n * pad
        self.box, self.s = box, box / n
        self.kernel_width = float(kernel_width)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = workspace_bytes(n, pad, kernel_width, max_particles)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        h = ctypes.c_void_p()
        rc = lib().mond_pm_create(Grid(n, pad), float(box), float(a0), float(G), int(mu_kind), float(kernel_width),
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.c_void_p(aligned),
                                  nbytes, int(max_particles), ctypes.byref(h))
        if rc != 0:
            raise MondError(rc, lib().mond_pm_last_error(None).decode())
        self.h = h
        self.particles = None

    # -- plumbing -----------------------------------------------------------
    def _check(self, rc: int):
        if rc != 0:
            raise MondError(rc, lib().mond_pm_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().mond_pm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C ABI, one method per entry point ------------------------------------
    def set_option(self, option: int, value: int):
        self._check(lib().mond_pm_set_option(self.h, int(option), int(value)))

    def bind_particles(self, cell, offset, vel, mass):
        """Borrow device tensors: cell int32 [N,3], offset float32 [N,3],
        vel float32 [N,3], mass float32 [N] (all contiguous)."""
        torch = self.torch
        for t, dt in ((cell, torch.int32), (offset, torch.float32), (vel, torch.float32), (mass, torch.float32)):
            if t.dtype != dt or not t.is_contiguous() or t.device != self.device:
                raise ValueError("particle tensors must be contiguous device tensors of the documented dtypes")
        self.particles = (cell, offset, vel, mass)
        self._check(lib().mond_pm_bind_particles(self.h, int(mass.numel()), _ptr(cell), _ptr(offset), _ptr(vel),
                                                 _ptr(mass)))

    def deposit(self):
        self._check(lib().mond_pm_deposit(self.h))

    def set_density(self, rho):
        """Mesh density (device float32 [n_f, n_f, n_f]) for the next solves."""
        self._check(lib().mond_pm_set_density(self.h, _ptr(rho)))

    def solve_field(self, n_iter: int = 4, warm: int = WARM_NONE, H_guess=None):
        self._check(lib().mond_pm_solve_field(self.h, int(n_iter), int(warm), _ptr(H_guess)))

    def smooth(self, out=None):
        self._check(lib().mond_pm_smooth(self.h, _ptr(out)))

    def gather_push(self, dt: float):
        self._check(lib().mond_pm_gather_push(self.h, float(dt)))

    def half_kick(self, dt: float):
        self._check(lib().mond_pm_half_kick(self.h, float(dt)))

    def gather(self, out=None):
        torch = self.torch
        N = self.particles[3].numel()
        if out is None:
            out = torch.empty((N, 3), dtype=torch.float32, device=self.device)
        self._check(lib().mond_pm_gather(self.h, _ptr(out)))
        return out

    def step(self, dt: float, n_iter: int = 4, warm: int = WARM_NONE):
        self._check(lib().mond_pm_step(self.h, float(dt), int(n_iter), int(warm)))

    def step_host(self, dt: float, n_iter: int, warm: int, cell_host, offset_host, vel_host):
        """Host tensors (pinned, contiguous) in and out; synchronises."""
        self._check(lib().mond_pm_step_host(self.h, float(dt), int(n_iter), int(warm), _ptr(cell_host),
                                            _ptr(offset_host), _ptr(vel_host)))

    def enable_increment(self, on: bool = True):
        """Attach (or detach) the workspace of the incremental solve
        (WARM_INCREMENT, Sect. 5.2 item v); later solves keep its base state."""
        lib().mond_pm_sync(self.h)  # nothing in flight may still use a released workspace
        if not on:
            self._check(lib().mond_pm_set_increment_workspace(self.h, None, 0))
            self.inc_workspace = None
            return
        n = ctypes.c_size_t()
        self._check(lib().mond_pm_increment_workspace_bytes(Grid(self.n, self.pad), ctypes.byref(n)))
        ws = self.torch.empty(n.value + 256, dtype=self.torch.uint8, device=self.device)
        aligned = (ws.data_ptr() + 255) & ~255
        self._check(lib().mond_pm_set_increment_workspace(self.h, ctypes.c_void_p(aligned), n.value))
        self.inc_workspace = ws

    def set_h_state(self, H):
        """Replace the warm-start H state by H (device float32 [3, n, n, n])."""
        if H.dtype != self.torch.float32 or not H.is_contiguous() or H.numel() != 3 * self.nf ** 3:
            raise ValueError("H must be a contiguous float32 tensor of 3 n^3 values")
        self._check(lib().mond_pm_set_h_state(self.h, _ptr(H)))

    def checkpoint(self, f, step: int = 0):
        """Write what a resumed run needs with torch.save: the bound particle
        arrays, the H state and the step count (synchronises)."""
        torch = self.torch
        H = self.get_field(FIELD_H)
        cell, off, vel, mass = self.particles
        state = {"nf": self.nf, "step": int(step), "cell": cell.cpu(), "offset": off.cpu(), "vel": vel.cpu(),
                 "mass": mass.cpu(), "H": H.cpu()}
        torch.save(state, f)

    def restore(self, f) -> int:
        """Load a checkpoint into the bound particle arrays and the H state;
        returns its step count. Replacing H drops the base of the incremental
        solve: a run of WARM_INCREMENT steps resumes with one full step."""
        torch = self.torch
        state = torch.load(f)
        if state["nf"] != self.nf or state["mass"].numel() != self.particles[3].numel():
            raise ValueError("checkpoint of another mesh or particle count")
        for dst, key in zip(self.particles, ("cell", "offset", "vel", "mass")):
            dst.copy_(state[key].to(self.device))
        H = state["H"].to(self.device).contiguous()
        torch.cuda.synchronize(self.device)  # torch's copies before the handle's stream reads them
        self.set_h_state(H)
        self.sync()
        return int(state["step"])

    def set_dipole_layer(self, axis: int, mass: float):
        """External field by a dipole layer of masses +-mass on the domain's end planes along axis (-1: none)."""
        self._check(lib().mond_pm_set_dipole_layer(self.h, int(axis), float(mass)))

    def density(self, which: int, out=None):
        """Density `which` (DENS_*) of the last solve's fields as [n, n, n] float32."""
        torch = self.torch
        if out is None:
            out = torch.empty((self.nf, self.nf, self.nf), dtype=torch.float32, device=self.device)
        self._check(lib().mond_pm_density(self.h, int(which), _ptr(out)))
        return out

    def shell_mass(self, which: int, center, dr: float, nbins: int) -> list:
        """Mass of density `which` in shells [k dr, (k+1) dr) about center (FP64, host)."""
        c = (_D * 3)(*[float(v) for v in center])
        out = (_D * int(nbins))()
        self._check(lib().mond_pm_shell_mass(self.h, int(which), c, float(dr), int(nbins), out))
        return list(out)

    def box_mass(self, which: int, lo, hi) -> float:
        """Mass in the box of cells lo..hi (inclusive, (x, y, z)) from the flux of the field."""
        a = (ctypes.c_int32 * 3)(*[int(v) for v in lo])
        b = (ctypes.c_int32 * 3)(*[int(v) for v in hi])
        out = _D(0.0)
        self._check(lib().mond_pm_box_mass(self.h, int(which), a, b, ctypes.byref(out)))
        return out.value

    def diagnostics(self) -> dict:
        d = Diag()
        self._check(lib().mond_pm_diagnostics(self.h, ctypes.byref(d)))
        return {"mass": d.mass, "momentum": list(d.momentum), "com": list(d.com), "ang_mom": list(d.ang_mom),
                "e_kin": d.e_kin, "e_pot": d.e_pot, "rho_mass": d.rho_mass, "n_iter_done": d.n_iter_done,
                "dH": list(d.dH)}

    def get_field(self, which: int, out=None):
        torch = self.torch
        planes = 3 if which in (FIELD_GN, FIELD_H, FIELD_ACC, FIELD_SMOOTH, FIELD_GM) else 1
        shape = (planes, self.nf, self.nf, self.nf) if planes == 3 else (self.nf, self.nf, self.nf)
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=self.device)
        self._check(lib().mond_pm_get_field(self.h, int(which), _ptr(out)))
        return out

    def field_ptr(self, which: int) -> int:
        """Device address of the handle's GN, H or ACC buffer (no copy, no sync)."""
        p = _P()
        self._check(lib().mond_pm_field_ptr(self.h, int(which), ctypes.byref(p)))
        return int(p.value)

    def get_deposit_acc(self):
        torch = self.torch
        out = torch.empty((self.nf, self.nf, self.nf), dtype=torch.int64, device=self.device)
        k = ctypes.c_int32(0)
        self._check(lib().mond_pm_get_deposit_acc(self.h, _ptr(out), ctypes.byref(k)))
        return out, int(k.value)

    def sync(self):
        self._check(lib().mond_pm_sync(self.h))

    def kernel_launches(self) -> int:
        return int(lib().mond_pm_kernel_launches(self.h))

    def kernel_stats(self) -> list:
        """Per kernel class since the last call (needs OPT_TIMING): name,
        launches, device ms, algorithmic bytes."""
        arr = (KStat * 32)()
        cnt = ctypes.c_int(0)
        self._check(lib().mond_pm_kernel_stats(self.h, arr, 32, ctypes.byref(cnt)))
        return [{"name": arr[i].name.decode(), "launches": int(arr[i].launches), "ms": float(arr[i].ms),
                 "bytes": float(arr[i].bytes)} for i in range(min(cnt.value, 32))]


def tune_key(h: MondPM, n_iter: int) -> str:
    """Key of a tuning result: the GPU, the FFT-domain side, the particle count
    (rounded to a power of two), the kernel width and the iteration count."""
    torch = h.torch
    n = h.particles[3].numel() if getattr(h, "particles", None) else 0
    return (f"{torch.cuda.get_device_name(h.device)}|nf={h.nf}|N~2^{max(n, 1).bit_length()}|"
            f"sigma={h.kernel_width:g}|K={int(n_iter)}")


def autotune(h: MondPM, n_iter: int = 4, trials: int = 3, cache: str | None = None):
    """Pick the work-item size and pass variant of one handle by timing
    zero-length steps (mond_pm_autotune); returns (chunk, pipelined). With a
    cache file (JSON), a result already stored for the same key is applied
    without timing, and a new result is stored."""
    import json
    import os

    key = tune_key(h, n_iter) if cache else None
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
        if key in table:
            chunk, pipelined = int(table[key]["chunk"]), int(table[key]["pipelined"])
            h.set_option(OPT_CHUNK, chunk)
            h.set_option(OPT_PIPELINED, pipelined)
            return chunk, pipelined
    c = ctypes.c_int64()
    p = ctypes.c_int()
    h._check(lib().mond_pm_autotune(h.h, int(n_iter), int(trials), ctypes.byref(c), ctypes.byref(p)))
    if cache:
        table[key] = {"chunk": int(c.value), "pipelined": int(p.value)}
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return int(c.value), int(p.value)


class Batch:
    """Independent systems stepped together as one CUDA graph per step
    (mond_pm_batch_*), replayed on the batch's stream. The handles stay owned
    by the caller; one that is also driven directly is synchronised first."""

    def __init__(self, handles, stream=None):
        import torch

        self.handles = list(handles)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        arr = (_P * len(self.handles))(*[h.h for h in self.handles])
        out = _P()
        rc = lib().mond_pm_batch_create(len(self.handles), arr, _P(self.stream.cuda_stream), ctypes.byref(out))
        if rc != 0:
            raise MondError(rc, lib().mond_pm_last_error(None).decode())
        self.b = out

    def step(self, dt: float, n_steps: int = 1, n_iter: int = 4, warm: int = WARM_NONE):
        rc = lib().mond_pm_batch_step(self.b, float(dt), int(n_steps), int(n_iter), int(warm))
        if rc != 0:
            raise MondError(rc, " / ".join(lib().mond_pm_last_error(h.h).decode() for h in self.handles[:1]))

    def sync(self):
        rc = lib().mond_pm_batch_sync(self.b)
        if rc != 0:
            raise MondError(rc, "device error in a batch member")

    def kernel_launches(self) -> int:
        return int(lib().mond_pm_batch_kernel_launches(self.b))

    def close(self):
        if getattr(self, "b", None):
            lib().mond_pm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
