"""B300-native explicit finite-difference time stepping (diffusion and acoustic
wave sweeps with damping, point sources and receivers) behind a C ABI.

The compute path is the CUDA library ``libfd_b300.so`` (include/fd.h); this
package only marshals arguments to it.  Importing the package does not load the
library; the first call does, and fails loudly if it has not been built.
"""

from .binding import (FD_ACOUSTIC, FD_DIFFUSION, FD_KERNEL_AUTO, FD_KERNEL_PLAIN,  # noqa: F401
                      FD_KERNEL_TMA, FdError, fd_create, fd_destroy, fd_kernel_launches, fd_kernel_name,
                      fd_last_error, fd_options_default, fd_profile, fd_read, fd_read_prev,
                      fd_reset, fd_run, fd_set_field, fd_set_model, fd_set_receivers, fd_set_sources,
                      fd_set_step, fd_stability_symbol, fd_steps_done, fd_version, fd_weights,
                      load, options)
from .binding import (fd_batch_add, fd_batch_create, fd_batch_destroy,  # noqa: F401
                      fd_batch_kernel_launches, fd_batch_remove, fd_batch_run, fd_batch_size,
                      fd_footprint_bytes)
from .solver import Batch, Solver  # noqa: F401

__all__ = ["Solver", "Batch", "FdError", "fd_batch_create", "fd_batch_add", "fd_batch_remove",
           "fd_batch_run", "fd_batch_size", "fd_batch_kernel_launches", "fd_batch_destroy",
           "fd_footprint_bytes", "fd_create", "fd_set_model", "fd_set_field", "fd_set_sources",
           "fd_set_receivers", "fd_run", "fd_read", "fd_read_prev", "fd_set_step", "fd_reset",
           "fd_steps_done", "fd_profile", "fd_kernel_name", "fd_kernel_launches", "fd_destroy", "fd_last_error",
           "fd_weights", "fd_stability_symbol", "fd_version", "fd_options_default", "options",
           "load"]
