"""Plain FP64 CPU oracle for the SMC / pCN-GM particle move (Lu, Jia, Meng,
"Sequential Monte Carlo with Gaussian Mixture Approximation for
Infinite-Dimensional Statistical Inverse Problems", arXiv 2503.16028).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, table or constant generator with the CUDA library under
``paper_2503_16028_gb300/csrc``; the two meet only through the seeded input
generators in ``paper_2503_16028_gb300/inputs.py`` (random arrays, no method
arithmetic) and through the Philox4x32-10 counter-based generator, which
each side implements on its own from its published definition.

Every function is written for a reader checking it against the paper by eye:
definitions written out, library primitives (matrix products, a sparse LU
solve, a banded solve) used as single steps, no blocking or fusion.

Modules
  philox   Philox4x32-10 uniforms and Box-Muller normals (random draws of
           Alg. 1 / Alg. 2; the paper names no generator).
  prior    Gaussian prior N(0, C), C = (I - alpha Lap)^-2, in its KL basis
           (Sec. 2.1, the trace-class prior; Sec. 3.2/3.1 for the operators).
  darcy    Forward model: steady Darcy flow -div(e^u grad w) = f, w = 0 on the
           boundary (Sec. 3.2, eq. example2:PDE), and the 1D analogue.
  observe  Point observations F(u) = (w(x_1), ..., w(x_Nd)) (Sec. 3.2) and the
           potential Phi(u) = |F(u) - d|^2 / (2 sigma^2) (Sec. 2.1).
  pcngm    pCN-GM proposal (Sec. 2.3, eq. pCN-GM proposal) and its
           acceptance ratio (eqs. auv of pCN-GMM, -GMM2 .. -GMM4, Thm 2).
  smc      Tempering by ESS bisection and the beta rule (App. C), reweighting,
           resampling and mutation of Alg. 1 / Alg. 3, posterior moments.
  gm       Gaussian-mixture fit on the leading KL modes (Sec. 2.4, the
           estimation step the paper delegates to its reference Feng2018).
  adjoint  dPhi/dx by the adjoint of the discrete forward model (the drift of
           the Langevin equation of App. B; Langevin kernels cited in Sec. 1
           and Sec. 2.4).
  langevin pCN-Langevin mutation: App. B's Langevin equation with the drift
           kept, Crank-Nicolson in the linear part, explicit drift.

Parity status: every function above is pinned by ``tests/test_oracle_*.py``
against closed forms, brute force or invariants; none is "parity unpinned".
"""
