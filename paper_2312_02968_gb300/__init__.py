"""GB300-native MOND particle-mesh force pipeline (Visser, Eijt & de Nijs 2023).

The compute path lives in the CUDA library ``libmondpm.so`` behind the C ABI of
``include/mond_pm.h`` (and ``include/mond_fno.h`` for the learned warm start);
``binding`` marshals arguments into it and nothing else. Importing this package
does not load the library; ``binding.lib()`` does, and raises if it has not
been built (``build.build()`` compiles it for sm_103a).

A time step of one system::

    import torch
    from paper_2312_02968_gb300 import binding as B, workloads as W

    p = W.isothermal(256, 1.0, 1_000_000, 8.0, 102.4, seed=1)   # cell, offset, vel, mass
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):               # the handle and torch's copies on one stream
        h = B.MondPM(256, 1, 256.0, 1.0, 1.0, B.MU_DEEP, 1.5, 1_000_000, stream=st)
        t = [torch.from_numpy(p[k]).cuda() for k in ("cell", "offset", "vel", "mass")]
        h.bind_particles(*t)
        h.set_option(B.OPT_USE_GRAPH, 1)      # each step one CUDA graph launch
        h.step(0.25, 4, B.WARM_NONE)          # deposit, 4 iterations, gather, kick, drift
        h.step(0.25, 1, B.WARM_PREV)          # warm start from the previous H
        phantom = h.density(B.DENS_PHANTOM)   # apparent minus baryonic density
        print(h.diagnostics()["e_kin"], phantom.sum().item())

Modules: ``binding`` (the handle, batches, the autotuner), ``surrogate`` and
``train_surrogate`` (the learned warm start), ``workloads`` (seeded initial
conditions), ``replicas`` (host logic of runs on several GPUs), ``build``.

Other warm starts: ``MOND_WARM_GUESS`` from the learned surrogate, and the
incremental solve of Sect. 5.2 (v) -- ``h.enable_increment()`` attaches its
workspace, a full step then keeps the base state, and ``h.step(dt, 1,
B.WARM_INCREMENT)`` iterates the linearised steps on the deposit's change.
"""
__all__ = ["binding", "workloads"]
