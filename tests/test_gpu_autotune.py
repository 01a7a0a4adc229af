"""The autotuner on the GPU: for every operation it times all candidate settings on the
caller's operands, keeps the fastest in its JSON cache, and the call made with the chosen
setting agrees with the oracle within the same gate as every other parity test."""
import json

import numpy as np
import pytest
import torch

import oracle
import spd_synth
import paper_2207_13901_gb300 as spd
from paper_2207_13901_gb300 import autotune
from tests._util import check_error, row_lengths

pytestmark = pytest.mark.gpu


def rounded(a, dtype):
    return torch.as_tensor(np.asarray(a, dtype=np.float64)).to(dtype).to(torch.float64).numpy()


def dev(a, dtype):
    return torch.as_tensor(np.asarray(a, dtype=np.float64)).to(dtype).cuda().contiguous()


def chosen(best):
    return {"split": best["split"], "tune": best["tune"]}


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_autotuned_settings_keep_parity(tmp_path, dtype):
    path = str(tmp_path / "tune.json")
    tuner = autotune.Autotuner(path=path, reps=1)
    rng = np.random.default_rng(31)
    A = spd_synth.rmat_csr(12, 16, seed=1)
    dA = spd.CSR.from_host(A.pos, A.crd, A.vals, (A.nrows, A.ncols), dtype=dtype)
    vr = rounded(A.vals, dtype)
    lens = row_lengths(A.pos)
    f64 = dtype == torch.float64

    x = rng.uniform(-1, 1, A.ncols)
    best = tuner.spmv(dA, dev(x, dtype))
    y = spd.spmv(dA, dev(x, dtype), **chosen(best))
    xr = rounded(x, dtype)
    check_error(y.double().cpu().numpy(), oracle.spmv(A.pos, A.crd, vr, xr, accurate=True),
                oracle.spmv(A.pos, A.crd, np.abs(vr), np.abs(xr)), f64, lens, "spmv %s" % best)

    for L in (16, 128):  # narrow L: the lane shapes are candidates too
        X = rng.uniform(-1, 1, (A.ncols, L))
        best = tuner.spmm(dA, dev(X, dtype))
        Y = spd.spmm(dA, dev(X, dtype), **chosen(best))
        Xr = rounded(X, dtype)
        check_error(Y.double().cpu().numpy(), oracle.spmm(A.pos, A.crd, vr, Xr, accurate=True),
                    oracle.spmm(A.pos, A.crd, np.abs(vr), np.abs(Xr)), f64, lens[:, None], "spmm L=%d %s" % (L, best))

    dY = rng.uniform(-1, 1, (A.nrows, 32))
    best = tuner.spmm_t(dA, dev(dY, dtype))
    dX = spd.spmm_t(dA, dev(dY, dtype), **chosen(best))
    dYr = rounded(dY, dtype)
    check_error(dX.double().cpu().numpy(), oracle.spmm_t(A.pos, A.crd, vr, dYr, A.ncols, accurate=True),
                oracle.spmm_t(A.pos, A.crd, np.abs(vr), np.abs(dYr), A.ncols), f64,
                np.bincount(A.crd, minlength=A.ncols)[:, None], "spmm_t %s" % best)

    K = 64
    C = rng.standard_normal((A.nrows, K))
    Dnk = rng.standard_normal((A.ncols, K))
    best = tuner.sddmm(dA, dev(C, dtype), dev(Dnk, dtype))
    out = spd.sddmm(dA, dev(C, dtype), dev(Dnk, dtype), **chosen(best))
    Cr, Dr = rounded(C, dtype), rounded(Dnk, dtype)
    check_error(out.double().cpu().numpy(), oracle.sddmm(A.pos, A.crd, vr, Cr, Dr, accurate=True),
                oracle.sddmm(A.pos, A.crd, np.abs(vr), np.abs(Cr), np.abs(Dr)), f64, K, "sddmm %s" % best, extra=1)

    T = spd_synth.zipf_csf3((300, 200, 400), 60000, 1.1, seed=3)
    dT = spd.CSF3.from_host(T.pos1, T.crd1, T.pos2, T.crd2, T.vals, T.dims, dtype=dtype)
    tv = rounded(T.vals, dtype)
    c = rng.standard_normal(T.dims[2])
    best = tuner.spttv(dT, dev(c, dtype))
    o = spd.spttv(dT, dev(c, dtype), **chosen(best))
    cr = rounded(c, dtype)
    check_error(o.double().cpu().numpy(), oracle.spttv(T.pos1, T.crd1, T.pos2, T.crd2, tv, cr, accurate=True),
                oracle.spttv(T.pos1, T.crd1, T.pos2, T.crd2, np.abs(tv), np.abs(cr)), f64, row_lengths(T.pos2),
                "spttv %s" % best)

    R = 32
    Cm = rng.standard_normal((T.dims[1], R))
    Dm = rng.standard_normal((T.dims[2], R))
    best = tuner.spmttkrp(dT, dev(Cm, dtype), dev(Dm, dtype))
    Am = spd.spmttkrp(dT, dev(Cm, dtype), dev(Dm, dtype), **chosen(best))
    Cmr, Dmr = rounded(Cm, dtype), rounded(Dm, dtype)
    sl = row_lengths(np.asarray(T.pos2, dtype=np.int64)[np.asarray(T.pos1, dtype=np.int64)])
    check_error(Am.double().cpu().numpy(),
                oracle.spmttkrp(T.pos1, T.crd1, T.pos2, T.crd2, tv, Cmr, Dmr, accurate=True),
                oracle.spmttkrp(T.pos1, T.crd1, T.pos2, T.crd2, np.abs(tv), np.abs(Cmr), np.abs(Dmr)), f64,
                sl[:, None], "spmttkrp %s" % best, extra=1)

    with open(path) as f:
        cache = json.load(f)
    ops = sorted({k.split("|")[0] for k in cache})
    assert ops == ["sddmm", "spmm", "spmm_t", "spmttkrp", "spmv", "spttv"]
    assert len(cache) == 7  # two SpMM widths
