"""FP64 CPU oracle for the D-GAMP-CT hot path (TEST INFRASTRUCTURE ONLY).

This package is a plain, slow, obviously-correct restatement of what the
paper (Perelli, Lexa, Can, Davies: "Compressive Computed Tomography
Reconstruction through Denoising Approximate Message Passing") computes in
each iteration of its Algorithm 1.  It exists to check the CUDA kernels: only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
leg of ``bench.py`` may import or run it.  The product path never routes
through it, and it shares no code with the CUDA library.

Modules, each citing the passage it follows:

* :mod:`oracle.geometry`     -- discretisation conventions (Section 2.1)
* :mod:`oracle.joseph`       -- system matrix A and its transpose (Eq. linCT)
* :mod:`oracle.precond`      -- Radon preconditioner V (Eqs. PPFT/Aprecon)
* :mod:`oracle.fanbeam`      -- flat-detector fan-beam A and Phi~ = A V^-1 (Section 6)
* :mod:`oracle.output_step`  -- Poisson output step, Laplace mode (Sec. 4.2, App. A)
* :mod:`oracle.tv`           -- proximal TV denoiser, l2 and (V^T V)^{-1} norms (Section 6.3)
* :mod:`oracle.philox`       -- counter-based probe generator for Eq. MC_SURE
* :mod:`oracle.gamp`         -- the D-GAMP-CT loop (Algorithm 1) and the
                                 i.i.d.-Gaussian GAMP used for state evolution
                                 (Section 3, Section 4.4)
* :mod:`oracle.cnn`          -- residual 3x3 CNN denoiser forward/backward
* :mod:`oracle.state_evolution` -- the scalar SE recursion for the CT slice (Section 4.4)

Everything runs in float64.  Functions whose result is not pinned to an
independent fact are marked "parity unpinned" in their docstring; at present
those are the full CT reconstruction (:func:`oracle.gamp.ct_solve`), which
the paper never reports on a synthetic input, and the state-evolution
recursion run on CT data (:func:`oracle.state_evolution.ct_state_evolution`),
whose recursion is pinned only through its i.i.d.-Gaussian reduction.
"""
