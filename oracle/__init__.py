"""FP64 CPU oracle for Joseph forward/back projection (paper Sec. 2.1-2.2),
listmode OSEM and the image-based resolution model (Sec. 2.6, 3, 4).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import or run anything in this
package.  It shares no code with the CUDA library and never imports it.

Every function here is pinned by ``tests/test_oracle_pins.py`` against
closed forms, brute force, invariants and hand-derived values; none is
"parity unpinned".
"""
from .joseph import (  # noqa: F401
    build, fwd, back, tof_weight, principal_axis, load, MODES,
)
from .osem import lm_osem_subset_update, lm_osem, poisson_loglik_grad, sino_osem_subset_update  # noqa: F401
from .resolution import gauss3d, gauss_taps, sigma_from_fwhm  # noqa: F401
