"""GB300-native sparse tensor algebra kernels of SpDISTAL (arXiv 2207.13901).

SpMV, SpMM, SpMM^T, SpAdd3, SDDMM, SpTTV and SpMTTKRP over CSR {Dense, Compressed} and CSF
{Dense, Compressed, Compressed} operands, split by rows (universe partition) or by
nonzeros (coordinate fusion + non-zero partition), executed by hand-written sm_103a
kernels behind the C ABI of include/spd.h. PyTorch supplies memory and streams.
"""
from .ops import (CSF3, CSR, ColumnBlocks, CSRTranspose, checked, column_blocks, csf3_workspace_size, csr_workspace_size,
                  fault_status, gather_vals, partition, result_dtype, sddmm, set_checked, spadd3, spadd3_numeric, spadd3_symbolic, spmm,
                  spmm_accumulate, spmm_column_blocked, spmm_t, spmttkrp, spmv, spttv, transpose, validate,
                  probe_bounded_wait)
from . import autograd, autotune, batched
from .batched import SpMMBatch

__all__ = ["CSR", "CSF3", "CSRTranspose", "spmv", "spmm", "spmm_t", "sddmm", "spttv", "spmttkrp", "validate",
           "partition", "set_checked", "checked", "transpose", "gather_vals", "spadd3", "spadd3_symbolic",
           "spadd3_numeric", "ColumnBlocks", "column_blocks", "spmm_accumulate", "spmm_column_blocked",
           "csr_workspace_size", "csf3_workspace_size", "result_dtype", "fault_status", "probe_bounded_wait", "autograd", "autotune", "batched", "SpMMBatch"]
