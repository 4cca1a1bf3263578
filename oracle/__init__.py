"""Plain FP64 CPU oracle for the batched Brinkmanlet swimmer forward model and TMCMC.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) may import, call, link or execute anything in this package.  It is
used by ``tests/``, by ``__graft_entry__.smoke()`` and by the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py``.  It shares no code with the CUDA path:
the only module both sides use is ``synthetic`` (seeded input generators, which
hold none of the method's arithmetic).

Modules
-------
brinkmanlet  regularized Brinkmanlet kernel functions (Sec. 2.1, Eqs. eqnblob, BrV)
swimmer      flagellum energies, forces, Euler stepping, observations, likelihood
             (Appendix Eqs. EFB, curva, EFT; Sec. 3.1 Eqs. likelihood, fitness)
tmcmc        transitional MCMC (Sec. 3.2, Algorithm 1) and delayed acceptance
mlp          FP64 reference MLP (forward, backward) for the learned surrogate

Parity status of every function is stated in its docstring: each is pinned by a
``-m "not gpu"`` test against a closed form, a library routine, an invariant or
brute force, except the end-to-end swimming trajectory, whose parity is
"parity unpinned" (the paper prints no trajectory values for these settings).
"""
