"""The fault path of the kernels' bounded waits, made to run out without a GPU fault.

The warp-tile SpMV/SpTTV kernels wait for their bulk copies with a wait bounded at 1 s,
after which they record a bit in a device fault word instead of spinning on. The probe
kernel waits, with the same code, for copies that are never issued, so its wait always
runs out; it touches nothing but its own shared memory and leaves no copy in flight.
The tests check that the host reads the fault (``spd_fault_status``, and checked mode
after a call), that reading clears it, and that the context keeps working."""
import time

import numpy as np
import pytest
import torch

import oracle
import spd_synth
import paper_2207_13901_gb300 as spd
from paper_2207_13901_gb300 import _abi
from tests._util import check_error, row_lengths

pytestmark = pytest.mark.gpu


def spmv_form2_against_oracle():
    A = spd_synth.rmat_csr(12, 16, seed=1)
    x = np.random.default_rng(3).uniform(-1, 1, A.ncols)
    dA = spd.CSR.from_host(A.pos, A.crd, A.vals, (A.nrows, A.ncols), dtype=torch.float32)
    xr = torch.as_tensor(x).float().double().numpy()
    vr = torch.as_tensor(A.vals).float().double().numpy()
    y = spd.spmv(dA, torch.as_tensor(x).float().cuda(), split="nnz", tune={"form": 2})
    check_error(y.double().cpu().numpy(), oracle.spmv(A.pos, A.crd, vr, xr, accurate=True),
                oracle.spmv(A.pos, A.crd, np.abs(vr), np.abs(xr)), False, row_lengths(A.pos), "spmv form 2")


def test_bounded_wait_runs_out_and_is_reported():
    assert spd.fault_status() == 0
    t0 = time.perf_counter()
    spd.probe_bounded_wait()
    flags = spd.fault_status()  # synchronizes the stream
    took = time.perf_counter() - t0
    assert flags == 1 and 0.9 < took < 60, (flags, took)
    assert spd.fault_status() == 0  # reading cleared it
    spmv_form2_against_oracle()  # the context still works, and the bulk-copy kernel completes its waits
    assert spd.fault_status() == 0


def test_checked_mode_reports_a_wait_that_ran_out():
    A = spd_synth.rmat_csr(10, 8, seed=2)
    dA = spd.CSR.from_host(A.pos, A.crd, A.vals, (A.nrows, A.ncols), dtype=torch.float32)
    x = torch.ones(A.ncols, device="cuda")
    spd.set_checked(True)
    try:
        spd.probe_bounded_wait()
        with pytest.raises(_abi.SpdError) as err:
            spd.spmv(dA, x, split="nnz", tune={"form": 2})  # checked mode reads the fault word after the call
        assert err.value.status == _abi.SPD_ERR_TIMEOUT
        spd.spmv(dA, x, split="nnz", tune={"form": 2})  # the next call starts clean
    finally:
        spd.set_checked(False)
    assert spd.fault_status() == 0
