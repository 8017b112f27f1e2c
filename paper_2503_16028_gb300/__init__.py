"""GB300 implementation of the SMC-pCN-GM particle move (arXiv 2503.16028).

Modules (none is imported here; importing the package loads neither torch nor
the CUDA library):

* ``smcgm``    -- ctypes binding of ``libsmcgm.so`` (the C ABI of include/smcgm.h)
                  and ``Sampler``, a context with its device workspace;
* ``autograd`` -- the potential Phi as a ``torch.autograd.Function`` (adjoint gradient);
* ``batch``    -- independent problems run concurrently, the solver-setting
                  autotuner, the mesh sweep and a per-layer JSON log of a run;
* ``exchange`` -- the host-side exchange of a layer split over ranks
                  (torch.distributed);
* ``inputs``   -- the synthetic workloads (presets, seeded observation points,
                  the stored data);
* ``build``    -- compiles ``libsmcgm.so`` for sm_103a in-tree with nvcc.
"""
