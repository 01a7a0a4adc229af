"""GPU parity of the batched persistent SpMM against the oracle, per matrix.

The batch mixes sizes (rows log-uniform, nnz per row uniform in [4, 64]) with
adversarial members: an empty matrix, a matrix without entries, one row longer than
4096 nonzeros. Every split policy and piece size is checked, and a CUDA-graph replay
after changing X and the values in place must produce the new products.
"""
import numpy as np
import pytest
import torch

import oracle
import spd_synth
import paper_2207_13901_gb300 as spd
from tests._util import check_error, row_lengths

pytestmark = pytest.mark.gpu



def rounded(a, dtype):
    return torch.as_tensor(np.asarray(a, dtype=np.float64)).to(dtype).to(torch.float64).numpy()


def make_batch(seed=0, count=24):
    mats = spd_synth.batched_uniform_csr(count, 1e2, 3e3, 4, 64, seed=seed)
    rng = np.random.default_rng(seed)
    mats.append(spd_synth.csr_from_coords(0, 5, [], [], vals=np.zeros(0)))            # no rows
    mats.append(spd_synth.csr_from_coords(40, 40, [], [], vals=np.zeros(0)))          # no entries
    big = np.sort(rng.choice(9000, 6000, replace=False))
    mats.append(spd_synth.csr_from_coords(9000, 9000, np.concatenate([np.full(6000, 17), np.arange(9000)]),
                                          np.concatenate([big, np.arange(9000)]),
                                          vals=rng.uniform(-1, 1, 15000)))           # one long row
    return mats


def check_batch(mats, Xs, Ys, dtype):
    for m, (A, X, Y) in enumerate(zip(mats, Xs, Ys)):
        if A.nrows == 0:
            continue
        vr, Xr = rounded(A.vals, dtype), rounded(X, dtype)
        ref = oracle.spmm(A.pos, A.crd, vr, Xr, accurate=True)
        scale = oracle.spmm(A.pos, A.crd, np.abs(vr), np.abs(Xr))
        check_error(Y.double().cpu().numpy(), ref, scale, dtype == torch.float64, row_lengths(A.pos)[:, None],
                    "matrix %d" % m)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float64])
@pytest.mark.parametrize("L", [64, 16, 7])
def test_batched_policies(dtype, L):
    mats = make_batch(1)
    rng = np.random.default_rng(2)
    Xh = [rng.uniform(-1, 1, (A.ncols, L)) for A in mats]
    dmats = [spd.CSR.from_host(A.pos, A.crd, A.vals, (A.nrows, A.ncols), dtype=dtype) for A in mats]
    Xs = [torch.as_tensor(X).to(dtype).cuda() for X in Xh]
    batch = spd.SpMMBatch(dmats, Xs)
    for policy, unit, threads in (("row", 64, 256), ("row", 1024, 256), ("nnz", 64, 256), ("nnz", 1024, 256),
                                  ("auto", 64, 256), ("auto", 1024, 256), ("nnz", 64, 512), ("auto", 1024, 64)):
        batch.configure(policy, unit, threads)
        for Y in batch.Ys:
            Y.fill_(float("nan"))
        batch.run()
        torch.cuda.synchronize()
        check_batch(mats, Xh, batch.Ys, dtype)
    # one launch per matrix gives the same products
    for Y in batch.Ys:
        Y.fill_(float("nan"))
    batch.run_separately()
    torch.cuda.synchronize()
    check_batch(mats, Xh, batch.Ys, dtype)


def test_batched_graph_replay_sees_new_values():
    dtype = torch.float32
    mats = make_batch(3, count=16)
    rng = np.random.default_rng(4)
    L = 64
    Xh = [rng.uniform(-1, 1, (A.ncols, L)) for A in mats]
    dmats = [spd.CSR.from_host(A.pos, A.crd, A.vals, (A.nrows, A.ncols), dtype=dtype) for A in mats]
    Xs = [torch.as_tensor(X).to(dtype).cuda() for X in Xh]
    batch = spd.SpMMBatch(dmats, Xs, policy="auto", unit_items=512)
    batch.capture()
    batch.replay()
    torch.cuda.synchronize()
    check_batch(mats, Xh, batch.Ys, dtype)
    # change X and the values in place: the captured graph must compute the new products
    Xh2 = [rng.uniform(-1, 1, (A.ncols, L)) for A in mats]
    for X, Xn in zip(Xs, Xh2):
        X.copy_(torch.as_tensor(Xn).to(dtype))
    mats2 = []
    for A, dA in zip(mats, dmats):
        v2 = rng.uniform(-1, 1, A.nnz)
        if A.nnz:
            dA.vals.copy_(torch.as_tensor(v2).to(dtype))
        mats2.append(spd_synth.CSR(A.nrows, A.ncols, A.pos, A.crd, v2))
    batch.replay()
    torch.cuda.synchronize()
    check_batch(mats2, Xh2, batch.Ys, dtype)


def test_batched_autotune_picks_a_valid_policy():
    dtype = torch.float32
    mats = make_batch(5, count=12)
    rng = np.random.default_rng(6)
    Xh = [rng.uniform(-1, 1, (A.ncols, 64)) for A in mats]
    dmats = [spd.CSR.from_host(A.pos, A.crd, A.vals, (A.nrows, A.ncols), dtype=dtype) for A in mats]
    batch = spd.SpMMBatch(dmats, [torch.as_tensor(X).to(dtype).cuda() for X in Xh])
    best = batch.autotune(units=(256, 1024), reps=2)
    assert best["policy"] in ("row", "nnz", "auto") and len(batch.tuning_table) == 6
    batch.run()
    torch.cuda.synchronize()
    check_batch(mats, Xh, batch.Ys, dtype)
