"""FP64 CPU oracle for the multi-species fast Fourier spectral collision operator.

Test infrastructure only.  Nothing in the product path (the CUDA library and its Python
binding) imports, links or executes anything in this package.  The only callers are
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py``.

The oracle follows the paper's own formulas step by step, in FP64, with no blocking,
fusion or symmetry reuse:

* ``quadrature``     -- radial Gauss-Legendre rule and spherical designs (Sec. 4).
* ``kernel``         -- nondimensional VSS/VHS prefactor (Eq. NVSS), domain rule
                        (Eq. domain), gain weight F and loss weight G^- (Eq. GG and
                        the loss-weight definition that follows it).
* ``fast_spectral``  -- truncated Fourier series, the fast gain sum and the loss
                        convolution of Sec. 4, evaluated literally for every ordered
                        species pair, radial node and design direction.
* ``direct``         -- the O(N^6) direct spectral sum (Eq. sum) with weights built by
                        brute-force sphere quadrature; used only to pin ``fast_spectral``.
* ``krook_wu``       -- the Krook-Wu exact solution of the homogeneous binary mixture
                        (Sec. 6.1) and its time derivative.
* ``moments``        -- macroscopic moments and the conservation residuals of Eq. consv.
* ``homogeneous``    -- SSP-RK2 time stepping of the homogeneous equation (Secs. 5, 6.1).
* ``dg1d``           -- nodal DG in one space dimension (Sec. 5): GLL rule, element matrices,
                        upwind transport, Maxwell walls (Sec. 2), the RKDG step.
"""

from . import quadrature, kernel, fast_spectral, direct, krook_wu, moments, homogeneous, dg1d  # noqa: F401
