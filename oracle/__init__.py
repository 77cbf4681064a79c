"""FP64 CPU oracle for the FLoD splatting path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. The product path (the CUDA library and its Python binding) never
imports it, and this package imports nothing from the product package: the two share no
code. Inputs come from the caller as numpy arrays (see the seeded generators), so the
oracle holds all of its own arithmetic.

Modules and the passages they follow:

* ``sh``          -- real spherical harmonics to degree 3 from the Legendre definition
                     (the colour model of Sec. 3, "spherical harmonic coefficients").
* ``gaussians``   -- Eq. 1 (covariance factorisation), Eq. 3 (level scale constraint),
                     Eq. 4 (constrained scale), Eq. 5 (AdjustScale), quaternion rotation.
* ``projection``  -- the projection to 2D of Eq. 2 (local affine / EWA), the
                     opacity-aware extent and the pixel/tile rectangles.
* ``raster``      -- binning into (tile, depth) keys, depth-ordered alpha blending
                     (Sec. 3, text after Eq. 2), the tiled and the brute-force per-pixel
                     renders, and the gradient (autograd of the written-out forward).
* ``select``      -- Eq. 6 (selective Gaussian set) and Eq. 7 (distance thresholds).
* ``loss``        -- the training loss of every level, L1 + D-SSIM (Sec. 5.1.4, the Loss
                     step of Algorithm 1), and its gradient.
* ``adam``        -- the Adam step of Algorithm 1 over one Gaussian set.
* ``prune``       -- overlap pruning (Sec. 4.3): the three nearest neighbours by brute force.
* ``densify``     -- density control (Densification and Pruning of Algorithm 1): the
                     2D-gradient statistics, clone, split and low-opacity pruning.

Parity status: every function above is pinned by ``tests/test_oracle_*.py`` against
closed forms, library routines, brute force, finite differences or values the paper
prints; none is "parity unpinned".
"""
from . import adam, densify, gaussians, loss, projection, prune, raster, select, sh  # noqa: F401
