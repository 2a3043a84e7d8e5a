"""FP64 CPU oracle of the two-population phase-field lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, readable
statement of what the GPU library computes, written from the paper
(Otomo, Zhang & Chen, "Improved phase-field-based lattice Boltzmann models
with a filtered collision operator", arXiv 1812.00118, Section 2 and Eq. 13).
Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The product path
(``paper_1812_00118_gb300``) never imports, links or runs anything here,
and nothing here imports the product path: the two share no code, no
tables and no helpers.

Modules
-------
lattice      D2Q9 / D3Q19 velocity sets and weights, lattice temperature T.
pflbm        the per-time-step update (Eqs. 1-14) on whole fields, FP64.
diagnostics  Laplace-law measurement and global sums used by validation.
surrogate    the learned warm start's convolutional network, forward and
             backward in FP64 (the reference of the tensor-core kernels).

Every function cites the section / equation it follows.  Readings of
places where the paper is silent or garbled are stated at the function
that takes them.  Parity status: every function here is pinned by
``tests/test_oracle_*.py``.  The diffusion correction ``delta_theta``
(Eq. 14) is pinned against what the mathematics fixes (it vanishes on the
tanh profile, leaves sum_i h^eq_i = phi, enters the first moment as
delta theta T n, and adds diffusion to a dense bubble); its function F is
this package's reading (R18 in ``pflbm``), since the paper leaves F open.
"""
