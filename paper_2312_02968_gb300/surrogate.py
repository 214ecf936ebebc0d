"""Learned warm start: a Fourier neural operator that maps the Newtonian field
g_N to the converged H of the MOND iteration (include/mond_fno.h).

The paper starts each solve from the previous step's H (Sect. 5.2, item iv).
Here the seed can instead come from the network, so that a single iteration
follows (MOND_WARM_GUESS). Training pairs are made by the solver itself:
a sphere-mixture density, its Newtonian field, and the H that the plain
iteration converges to. Everything below is argument marshalling and host
control flow; the arithmetic runs in the CUDA library.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import binding as B
from .binding import FnoShape, MondError, lib

DEFAULT_SHAPE = (64, 32, 16, 4)  # coarse side, width, modes per axis, layers
REF_ITERS = 40  # converged reference: mean of iterates 40 and 41 (the undamped scheme ends in a 2-cycle)


def _p(t):
    """Tensor or raw device address -> void*."""
    if t is None:
        return None
    return ctypes.c_void_p(t) if isinstance(t, int) else ctypes.c_void_p(t.data_ptr())


def _check(rc, what):
    if rc != 0:
        raise MondError(rc, what)


class FNO:
    """Parameters, Adam state and workspace of one network on one device."""

    def __init__(self, n=64, width=32, modes=16, layers=4, seed=0, device=None, stream=None):
        import torch

        self.torch = torch
        self.shape = FnoShape(n, width, modes, layers)
        self.n = n
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        cnt = ctypes.c_int64()
        _check(lib().mond_fno_param_count(self.shape, ctypes.byref(cnt)), "unsupported FNO shape")
        self.count = int(cnt.value)
        ws = ctypes.c_size_t()
        _check(lib().mond_fno_workspace_bytes(self.shape, ctypes.byref(ws)), "unsupported FNO shape")
        f32 = dict(dtype=torch.float32, device=self.device)
        self.params = torch.empty(self.count, **f32)
        self.params_bf16 = torch.empty(self.count, dtype=torch.int16, device=self.device)
        self.grad = torch.zeros(self.count, **f32)
        self.m = torch.zeros(self.count, **f32)
        self.v = torch.zeros(self.count, **f32)
        self.ws = torch.empty(int(ws.value) + 256, dtype=torch.uint8, device=self.device)
        self.ws_ptr = ctypes.c_void_p((self.ws.data_ptr() + 255) & ~255)
        self.loss_acc = torch.zeros(2, dtype=torch.float64, device=self.device)
        self.adam_scratch = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.steps = 0
        self.init(seed)

    @property
    def _st(self):
        return ctypes.c_void_p(self.stream.cuda_stream)

    def init(self, seed: int):
        _check(lib().mond_fno_init(self.shape, ctypes.c_uint64(seed), _p(self.params), self._st), "init")
        self.cast()

    def cast(self):
        _check(lib().mond_fno_cast(self.shape, _p(self.params), _p(self.params_bf16), self._st), "cast")

    def load(self, params):
        self.params.copy_(params)
        self.cast()

    def forward(self, x, y):
        """x [4, n, n, n] -> y [3, n, n, n] (float32, device)."""
        _check(lib().mond_fno_forward(self.shape, _p(self.params_bf16), _p(x), _p(y), self.ws_ptr, self._st),
               "forward")
        return y

    def backward(self, x, dy):
        """Gradient of the sample of the last forward, added into self.grad."""
        _check(lib().mond_fno_backward(self.shape, _p(self.params_bf16), _p(x), _p(dy), _p(self.grad),
                                       self.ws_ptr, self._st), "backward")

    def loss(self, y, t, dy, weight=1.0):
        _check(lib().mond_fno_loss(int(y.numel()), _p(y), _p(t), _p(dy), float(weight), _p(self.loss_acc),
                                   self._st), "loss")

    def adam(self, lr, b1=0.9, b2=0.999, eps=1e-8, clip=0.0):
        """One Adam step; clip > 0 caps the gradient norm; a non-finite
        gradient is dropped."""
        self.steps += 1
        _check(lib().mond_fno_adam(self.count, _p(self.params), _p(self.grad), _p(self.m), _p(self.v), float(lr),
                                   float(b1), float(b2), float(eps), self.steps, float(clip), _p(self.adam_scratch),
                                   self._st), "adam")
        self.cast()

    # ----------------------------------------------------------- training
    def train(self, xs, ts, epochs: int, batch: int, lr: float, seed: int = 0, lr_final: float | None = None,
              log=None, clip: float = 5.0):
        """Adam on the relative squared error over pairs xs [P, 4, n^3], ts
        [P, 3, n^3] (device); cosine-decayed learning rate. Returns the mean
        loss of each epoch."""
        torch = self.torch
        P = xs.shape[0]
        y = torch.empty_like(ts[0])
        dy = torch.empty_like(ts[0])
        rng = np.random.default_rng(seed)
        total = epochs * max(1, P // batch)
        lr_final = lr * 0.05 if lr_final is None else lr_final
        hist = []
        it = 0
        for ep in range(epochs):
            order = rng.permutation(P)
            self.loss_acc.zero_()
            nb = max(1, P // batch)
            for b in range(nb):
                for i in order[b * batch:(b + 1) * batch]:
                    self.forward(xs[i], y)
                    self.loss(y, ts[i], dy, 1.0 / batch)
                    self.backward(xs[i], dy)
                cur = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * it / max(1, total - 1)))
                self.adam(cur, clip=clip)
                it += 1
            hist.append(float(self.loss_acc[0].item()) / nb)
            if log:
                log(f"epoch {ep}: loss {hist[-1]:.4e}")
        return hist


# ---------------------------------------------------------- field mappings
def features(gN, N: int, n: int, a0: float, x, scale, stream):
    """Network input x [4, n^3] and scale (4 floats, device) from g_N [3, N^3]."""
    _check(lib().mond_fno_input(N, n, float(a0), _p(gN), _p(x), _p(scale), ctypes.c_void_p(stream.cuda_stream)),
           "input")


def upsample(y, N: int, n: int, scale, H, stream, scratch=None):
    """H [3, N^3] = scale * cubic upsampling of y [3, n^3]; scratch: a device
    uint8 tensor of at least mond_fno_output_scratch_bytes(N, n) bytes (made
    here when not given)."""
    if scratch is None:
        import torch

        scratch = torch.empty(int(lib().mond_fno_output_scratch_bytes(N, n)), dtype=torch.uint8, device=H.device)
    _check(lib().mond_fno_output(N, n, _p(y), _p(scale), _p(H), _p(scratch), ctypes.c_void_p(stream.cuda_stream)),
           "output")


def coarsen(fine, N: int, n: int, ncomp: int, coarse, scale, stream, fine2=None):
    _check(lib().mond_fno_coarsen(N, n, ncomp, _p(fine), _p(fine2), _p(coarse), _p(scale),
                                  ctypes.c_void_p(stream.cuda_stream)), "coarsen")


def mixture_density(N: int, s: float, spheres: dict, rmax: float, rho, stream):
    """Mesh density of a sphere mixture (dict of numpy arrays: centre [K, 3]
    in pixels from the domain centre, mass [K], radius [K] pixels, kind [K])."""
    import torch

    dev = rho.device
    c = torch.as_tensor(np.asarray(spheres["centre"], np.float32).reshape(-1), device=dev)
    m = torch.as_tensor(np.asarray(spheres["mass"], np.float32), device=dev)
    r = torch.as_tensor(np.asarray(spheres["radius"], np.float32), device=dev)
    k = torch.as_tensor(np.asarray(spheres["kind"], np.int32), device=dev)
    _check(lib().mond_fno_mixture_density(N, float(s), int(m.numel()), _p(c), _p(m), _p(r), _p(k), float(rmax),
                                          _p(rho), ctypes.c_void_p(stream.cuda_stream)), "mixture density")
    return (c, m, r, k)  # keep the inputs alive until the stream has used them


def converged_H(h: "B.MondPM", zeros, Ha, Hb):
    """H at iterates REF_ITERS and REF_ITERS + 1 from H = 0 (the current
    density of h): Ha, Hb [3, n^3] device."""
    h.solve_field(REF_ITERS, B.WARM_GUESS, zeros)
    h.get_field(B.FIELD_H, Ha)
    h.solve_field(1, B.WARM_PREV)
    h.get_field(B.FIELD_H, Hb)


def make_pairs(h: "B.MondPM", fno_n: int, seeds, a0: float, sphere_params, log=None):
    """Training pairs from the solver: for each seed a mixture density, x =
    features(g_N), t = coarse converged H / scale. Returns (xs, ts)."""
    import torch

    nf, st = h.nf, h.stream
    dev = h.device
    P = len(seeds)
    V = fno_n ** 3
    xs = torch.empty((P, 4, V), dtype=torch.float32, device=dev)
    ts = torch.empty((P, 3, V), dtype=torch.float32, device=dev)
    rho = torch.empty(nf ** 3, dtype=torch.float32, device=dev)
    zeros = torch.zeros(3 * nf ** 3, dtype=torch.float32, device=dev)
    Ha = torch.empty(3 * nf ** 3, dtype=torch.float32, device=dev)
    Hb = torch.empty_like(Ha)
    gN = torch.empty_like(Ha)
    scale = torch.empty(4, dtype=torch.float32, device=dev)
    with torch.cuda.stream(st):
        for i, sd in enumerate(seeds):
            sp = sphere_params(nf, sd)
            keep = mixture_density(nf, h.s, sp, 0.4 * nf, rho, st)
            h.set_density(rho)
            converged_H(h, zeros, Ha, Hb)
            h.get_field(B.FIELD_GN, gN)
            features(gN, nf, fno_n, a0, xs[i], scale, st)
            coarsen(Ha, nf, fno_n, 3, ts[i], scale, st, fine2=Hb)
            del keep
            if log and (i + 1) % 100 == 0:
                log(f"pairs {i + 1}/{P}")
    h.sync()
    return xs, ts


class GuessSolver:
    """Learned warm start on one handle: Newton solve, network input from g_N,
    forward pass, upsampling to the mesh, then MOND_WARM_GUESS with n_iter
    iterations. All launches go to the handle's stream; no synchronisation."""

    def __init__(self, h: "B.MondPM", net: FNO, a0: float):
        import torch

        if net.stream.cuda_stream != h.stream.cuda_stream:
            raise ValueError("the network and the handle must share one stream")
        self.h, self.net, self.a0 = h, net, a0
        n, nf = net.n, h.nf
        dev = h.device
        self.x = torch.empty((4, n, n, n), dtype=torch.float32, device=dev)
        self.y = torch.empty((3, n, n, n), dtype=torch.float32, device=dev)
        self.scale = torch.empty(4, dtype=torch.float32, device=dev)
        self.H = torch.empty((3, nf, nf, nf), dtype=torch.float32, device=dev)
        self.up_scratch = torch.empty(int(lib().mond_fno_output_scratch_bytes(nf, n)), dtype=torch.uint8,
                                      device=dev)
        self.gN = h.field_ptr(B.FIELD_GN)

    def predict(self):
        """H guess of the current density into self.H (after a Newton solve)."""
        h, net = self.h, self.net
        h.solve_field(0, B.WARM_NONE)
        features(self.gN, h.nf, net.n, self.a0, self.x, self.scale, h.stream)
        net.forward(self.x, self.y)
        upsample(self.y, h.nf, net.n, self.scale, self.H, h.stream, self.up_scratch)
        return self.H

    def solve(self, n_iter: int = 1, project: bool = False):
        """predict() then n_iter iterations from the guess (projected onto its
        divergence-free part first when project is set); the Newton field of
        predict() is reused by the solve."""
        self.predict()
        self.h.solve_field(n_iter, B.WARM_GUESS if project else B.WARM_GUESS_RAW, self.H)
