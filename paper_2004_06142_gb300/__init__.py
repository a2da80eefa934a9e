"""GB300-native PNOF5 / PNOF7 / PNOF7s energy and orbital-Lagrangian build (arXiv:2004.06142).

The compute path is libdonof.so (CUDA for sm_103a, C ABI in include/donof.h); this
package holds its build script and a thin ctypes binding.
"""
from .binding import (  # noqa: F401
    B_DENSE, B_PACKED, BATCH_BACKWARD, BATCH_GRAPH, BATCH_STREAMS, FP64, MIXED, PNOF5, PNOF7, PNOF7S, Batch, Builder, DonofEnergy, DonofError,
    donof_batched_workspace_size, donof_energy_backward, donof_energy_lagrangian, donof_energy_lagrangian_noalloc, donof_noalloc_read_status, donof_get_jk, donof_nofmp2_static, donof_partial_size, donof_energy_lagrangian_partial, donof_energy_lagrangian_finish, shard_range, exchange_partial, donof_optimize_occupations, donof_orbital_update, donof_eigh, donof_eigh_read_status, donof_host_staging_size, donof_energy_lagrangian_host, alloc_workspace, donof_prepare_B,
    donof_launch_count, donof_profile_enable, donof_profile_read,
    donof_read_status, donof_status_string, PHASES, donof_workspace_size, energy, make_problem,
)
