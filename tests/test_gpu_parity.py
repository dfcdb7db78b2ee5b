"""GPU parity: every C-ABI call against the oracle on the same seeded inputs.

FP64 mode: results agree with the oracle to rounding (1e-10 relative on
gauge-invariant quantities: dense reconstructions, norms, C_eff). The random
sketches are generated from the same Philox stream on both sides."""
import numpy as np
import pytest

from oracle import dense, qtt as oq
from paper_2412_11566_gb300 import synth
from tests._helpers import from_lib_op, random_tt, to_lib_op

pytestmark = pytest.mark.gpu

SEED = 2412


@pytest.fixture(scope="module")
def Q(lib_built):
    return lib_built


@pytest.fixture(scope="module")
def ctx64(Q):
    c = Q.Context(0, Q.QTT_FP64, 1 << 30, seed=SEED)
    yield c
    c.close()


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def qtt_dims(n):
    return [6] + [2] * (3 * n)


def test_tt_roundtrip(Q, ctx64):
    rng = np.random.default_rng(0)
    x = random_tt(rng, qtt_dims(2), [1, 3, 5, 4, 6, 3, 2, 1])
    t = ctx64.tt(x)
    y = t.cores()
    for a, b in zip(x, y):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tt_to_dense_vs_oracle(Q, precision):
    """qtt_tt_to_dense against the oracle's contraction of the same cores
    (eq. (tt_format)), on the values each context holds."""
    prec = Q.QTT_FP64 if precision == "fp64" else Q.QTT_FP32
    ctx = Q.Context(0, prec, 1 << 28, seed=SEED)
    try:
        rng = np.random.default_rng(9)
        x = random_tt(rng, qtt_dims(3), [1, 6, 12, 20, 17, 14, 11, 8, 4, 2, 1])
        if precision == "fp32":
            x = [c.astype(np.complex64).astype(np.complex128) for c in x]
        got = ctx.tt(x).to_dense()
        ref = oq.tt_full(x)
        assert got.shape == ref.shape
        assert rel(got, ref) < (1e-13 if precision == "fp64" else 1e-6)
    finally:
        ctx.close()


@pytest.mark.parametrize("n,ranks", [(2, [1, 6, 9, 12, 10, 7, 2, 1]), (3, [1, 6, 12, 20, 17, 14, 11, 8, 4, 2, 1])])
def test_round_vs_oracle(Q, ctx64, n, ranks):
    rng = np.random.default_rng(n)
    x = random_tt(rng, qtt_dims(n), ranks)
    full = oq.tt_full(x)
    for eps, rmax in [(1e-12, 1000), (1e-2, 1000), (0.3, 1000), (1e-12, 5)]:
        t = ctx64.tt(x)
        rc = Q.tt_round(ctx64, t, eps, rmax)
        y = t.cores()
        ref, cap = oq.tt_round(x, eps, rmax)
        assert [c.shape for c in y] == [c.shape for c in ref]
        assert rc == (Q.QTT_WRANKCAP if cap else 0)
        assert rel(oq.tt_full(y), oq.tt_full(ref)) < 1e-10
        if rmax == 1000:
            assert rel(oq.tt_full(y), full) <= eps * (1 + 1e-9)
        # right-orthogonal result
        for c in y[1:]:
            M = c.reshape(c.shape[0], -1)
            assert np.abs(M @ M.conj().T - np.eye(M.shape[0])).max() < 1e-11


def test_dot_and_norm(Q, ctx64):
    rng = np.random.default_rng(5)
    a = random_tt(rng, qtt_dims(2), [1, 4, 6, 5, 6, 4, 3, 1])
    b = random_tt(rng, qtt_dims(2), [1, 3, 5, 7, 5, 4, 2, 1])
    got = Q.qtt_tt_dot(ctx64, ctx64.tt(a), ctx64.tt(b))
    ref = np.vdot(oq.tt_full(a), oq.tt_full(b))
    assert abs(got - ref) < 1e-11 * abs(ref)


@pytest.mark.parametrize("n", [2, 3])
def test_sketched_apply_vs_oracle(Q, ctx64, n):
    rng = np.random.default_rng(10 + n)
    lam0, mu0 = 2.0, 1.0
    G = oq.gamma_qtt(n, lam0, mu0, 1e-12)
    S = oq.sfft_operator(n)
    x = random_tt(rng, qtt_dims(n), [1] + [min(6 * 2 ** k, 2 ** (3 * n - k), 9) for k in range(3 * n)] + [1])
    x, _ = oq.tt_round(x, 1e-14, 1000)
    tx = ctx64.tt(x)
    for op, name in [(G, "gamma"), (S, "sfft")]:
        cores, diag = to_lib_op(op)
        top = ctx64.op(cores, diag)
        for rmax, eps in [(200, 1e-12), (12, 1e-12), (200, 1e-3)]:
            y, rc = Q.qtt_op_apply(ctx64, top, tx, eps, rmax, 16, apply_id=7)
            ref = oq.tto_apply_sketched(op, x, rmax + 16, SEED, 7)
            ref, cap = oq.tt_round(ref, eps, rmax, assume_left_orth=True)
            yc = y.cores()
            assert [c.shape for c in yc] == [c.shape for c in ref], name
            assert rel(oq.tt_full(yc), oq.tt_full(ref)) < 1e-10, (name, rmax, eps)
            if rmax == 200 and eps == 1e-12:
                exact = oq.tto_full(op) @ oq.tt_full(x).reshape(-1)
                assert rel(oq.tt_full(yc).reshape(-1), exact) < 1e-10


@pytest.mark.parametrize("n", [2, 3])
def test_sfft_operator_vs_oracle(Q, ctx64, n):
    for adj in (False, True):
        op = Q.qtt_sfft_operator(ctx64, n, adj, 1e-14)
        cores, diag = op.cores(), op.shape()[3]
        ref = oq.sfft_operator(n, 1e-14, adjoint=adj)
        assert rel(oq.tto_full(from_lib_op(cores, diag)), oq.tto_full(ref)) < 1e-12


@pytest.mark.parametrize("n", [2, 3])
def test_gamma_operator_vs_oracle(Q, ctx64, n):
    # two reference media from the same cached monomial TT (the separable
    # construction), each against the oracle's TT-SVD of its own Green field
    for lam0, mu0 in [(3.5, 1.25), (0.7, 4.0)]:
        op = Q.qtt_gamma_operator(ctx64, n, lam0, mu0, 0, 1e-12)
        cores, diag = op.cores(), op.shape()[3]
        G = oq.tto_full(from_lib_op(cores, diag))
        ref = oq.tto_full(oq.gamma_qtt(n, lam0, mu0, 1e-12))
        assert rel(G, ref) < 1e-9


def test_stiffness_operator_vs_oracle(Q, ctx64):
    n = 3
    ph = synth.centred_sphere(n, 0.3)
    E, nu = (1.0, 10.0), (0.3, 0.25)
    lam0 = dense.reference_lame(E, nu)
    op = Q.qtt_from_phase_field(ctx64, ph, n, E, nu, None, 1e-12)
    got = oq.tto_full(from_lib_op(op.cores(), op.shape()[3]))
    ref = oq.tto_full(oq.stiffness_qtt(ph, n, E, nu, lam0, 1e-12))
    assert rel(got, ref) < 1e-10


def test_stiffness_operator_broadcast_axis(Q, ctx64):
    n = 3
    ph = synth.laminate(n, 2)          # shape (1, 1, 8): broadcast x1, x2
    E, nu = (1.0, 5.0), (0.3, 0.3)
    lam0 = dense.reference_lame(E, nu)
    op = Q.qtt_from_phase_field(ctx64, ph, n, E, nu, None, 1e-12)
    got = oq.tto_full(from_lib_op(op.cores(), op.shape()[3]))
    ref = oq.tto_full(oq.stiffness_qtt(synth.broadcast_dense(ph, n), n, E, nu, lam0, 1e-12))
    assert rel(got, ref) < 1e-10


@pytest.mark.parametrize("nphase", [3, 40])
def test_phase_matrices_operator_vs_oracle(Q, ctx64, nphase):
    """Arbitrary (non-isotropic) phase matrices: 3 phases take the reduced
    path (field = U Y with the 36-row Voigt range of the 3 matrices), 40
    phases exceed 36 and take the full 36-row field."""
    n = 2
    rng = np.random.default_rng(SEED + nphase)
    ph = rng.integers(0, nphase, size=(4, 4, 4)).astype(np.uint8)
    mats = rng.standard_normal((nphase, 6, 6))
    op = Q.qtt_from_phase_matrices(ctx64, ph, n, mats, 1e-12)
    got = oq.tto_full(from_lib_op(op.cores(), op.shape()[3]))
    ref = oq.tto_full(oq.phase_matrices_qtt(ph, n, mats, 1e-12))
    assert rel(got, ref) < 1e-10


def test_operators_through_gram_path(Q):
    """Every dense-field TT-SVD unfolding through the Gram path (threshold
    0): the tall-skinny Gram and M V kernels for narrow bonds, the tiled
    GEMM for wide ones."""
    ctx = Q.Context(0, Q.QTT_FP64, 1 << 30, seed=SEED)
    try:
        ctx.set_tt_svd(0.0)
        n = 3
        ph = synth.centred_sphere(n, 0.3)
        E, nu = (1.0, 10.0), (0.3, 0.25)
        lam0 = dense.reference_lame(E, nu)
        op = Q.qtt_from_phase_field(ctx, ph, n, E, nu, None, 1e-10)
        got = oq.tto_full(from_lib_op(op.cores(), op.shape()[3]))
        ref = oq.tto_full(oq.stiffness_qtt(ph, n, E, nu, lam0, 1e-12))
        assert rel(got, ref) < 1e-9
        g = Q.qtt_gamma_operator(ctx, n, 3.5, 1.25, 0, 1e-10)
        got = oq.tto_full(from_lib_op(g.cores(), g.shape()[3]))
        ref = oq.tto_full(oq.gamma_qtt(n, 3.5, 1.25, 1e-12))
        assert rel(got, ref) < 1e-9
        with pytest.raises(Q.QttError):
            ctx.set_tt_svd(-1.0)
    finally:
        ctx.close()


def test_mean_vs_dense(Q, ctx64):
    n = 2
    rng = np.random.default_rng(3)
    ph = synth.centred_sphere(n, 0.3)
    E, nu = (1.0, 4.0), (0.3, 0.2)
    lam0 = dense.reference_lame(E, nu)
    dC = oq.stiffness_qtt(ph, n, E, nu, lam0, 1e-12)
    x = random_tt(rng, qtt_dims(n), [1, 6, 5, 4, 6, 4, 2, 1])
    cores, diag = to_lib_op(dC)
    got = Q.qtt_op_mean_apply(ctx64, ctx64.op(cores, diag), ctx64.tt(x))
    ref = (oq.tto_full(dC) @ oq.tt_full(x).reshape(-1)).reshape(6, -1).mean(axis=1)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def tie_free_tol(history, m):
    """A stop tolerance between the residuals of iterations m-1 and m: both
    sides then stop after exactly m iterations (the GPU's residual uses FP64
    inner products, whose cancellation floor is ~1e-8 relative, so a tolerance
    within that band of a residual could flip the decision)."""
    return float(np.sqrt(history[m - 2] * history[m - 1]))


@pytest.mark.parametrize("n,load,m", [(2, 0, 20), (2, 4, 12), (3, 0, 8), (3, 3, 6)])
def test_ls_solve_ops_vs_qtt_oracle(Q, ctx64, n, load, m):
    ph = synth.centred_sphere(n, 0.3)
    E, nu = (1.0, 10.0), (0.3, 0.3)
    lam0 = dense.reference_lame(E, nu)
    eps, rmax = 1e-8, 24
    dC = oq.stiffness_qtt(ph, n, E, nu, lam0, 1e-12)
    G = oq.gamma_qtt(n, *lam0, 1e-12)
    S, Sh = oq.sfft_operator(n), oq.sfft_operator(n, adjoint=True)
    C0 = dense.stiffness_voigt(*lam0)
    Ev = np.eye(6)[load]
    ref = oq.ls_solve(dC, G, S, Sh, Ev, n, 1e-300, eps, rmax, max_iter=m, lame0=lam0, seed=SEED)
    tol = tie_free_tol(ref["history"], m)
    dc, dd = to_lib_op(dC)
    gc, gd = to_lib_op(G)
    sig, info, rc = Q.ls_solve_ops(ctx64, ctx64.op(dc, dd), ctx64.op(S), ctx64.op(Sh),
                                   ctx64.op(gc, gd), C0, Ev, Q.solve_params(tol, 500, eps, rmax))
    assert info["iters"] == m
    assert abs(info["residual"] - ref["history"][-1]) < 1e-6 * ref["history"][-1] + 1e-12
    assert np.abs(sig - ref["sigma_bar"]).max() < 1e-10 * np.abs(ref["sigma_bar"]).max()


def test_ls_solve_vs_dense_oracle(Q, ctx64):
    """Operators built on the device (phase field, SFFT, Green) and the full
    solve against the dense FFT scheme (Alg. 1)."""
    n = 3
    ph = synth.centred_sphere(n, 0.3)
    E, nu = (1.0, 10.0), (0.3, 0.3)
    dC = Q.qtt_from_phase_field(ctx64, ph, n, E, nu, None, 1e-10)
    C, infos, rc = Q.ls_solve_ceff(ctx64, dC, Q.solve_params(1e-6, 500, 1e-9, 64), loads=[0, 3])
    Cd, imag, its = dense.ceff(ph, E, nu, tol=1e-6, loads=[0, 3])
    for k in (0, 3):
        assert np.abs(C[:, k] - Cd[:, k]).max() < 1e-5 * np.abs(Cd).max()


def test_fp32_mode_vs_dense_oracle(Q):
    """FP32 mode (complex64 cores, FP32 contractions and factorisations, FP64
    norms and C_eff average) against the tightly converged dense oracle:
    7.6e-6 relative measured on this contrast-10 case (the FP32 residual floor
    keeps the iteration from reaching tol 1e-6, so it runs to the cap)."""
    ctx = Q.Context(0, Q.QTT_FP32, 1 << 30, seed=SEED)
    n = 3
    ph = synth.centred_sphere(n, 0.3)
    E, nu = (1.0, 10.0), (0.3, 0.3)
    dC = Q.qtt_from_phase_field(ctx, ph, n, E, nu, None, 1e-6)
    C, infos, rc = Q.ls_solve_ceff(ctx, dC, Q.solve_params(1e-6, 500, 1e-6, 64), loads=[0, 3])
    Cd, imag, its = dense.ceff(ph, E, nu, tol=1e-10, loads=[0, 3])
    for k in (0, 3):
        assert np.abs(C[:, k] - Cd[:, k]).max() < 5e-5 * np.abs(Cd).max()
    ctx.close()


def test_fp32_mode_eight_spheres_16(Q):
    """The benchmark's 8-sphere geometry (contrast 20) at 16^3, FP32 mode at
    the workload's settings (tol 1e-4, eps_tt 1e-6, r_max 128, which is the
    full rank at this size): converges like FP64 (29 iterations) and meets the
    1e-4 C_eff goal against the dense oracle (4.8e-5 measured). Before the
    sketch environments were orthonormalised FP32 stalled at a 1e-2 residual."""
    w = synth.spheres256(n=4)
    ctx = Q.Context(0, Q.QTT_FP32, 4 << 30, seed=SEED)
    try:
        dC = Q.qtt_from_phase_field(ctx, w.phase, w.n, w.E, w.nu, None, w.eps_tt, w.rmax)
        C, infos, rc = Q.ls_solve_ceff(ctx, dC, Q.solve_params(w.tol, 80, w.eps_tt, w.rmax),
                                       loads=[0])
        Cd, imag, its = dense.ceff(w.phase, w.E, w.nu, tol=1e-8, loads=[0])
        assert infos[0]["iters"] < 40 and infos[0]["residual"] < w.tol
        assert np.abs(C[:, 0] - Cd[:, 0]).max() < 1e-4 * np.abs(Cd).max()
    finally:
        ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_concurrent_loads_match_sequential(Q, precision):
    """Six load cases on six streams/lanes give the same C_eff as one after
    the other (same sketches, same operators)."""
    prec = Q.QTT_FP64 if precision == "fp64" else Q.QTT_FP32
    ctx = Q.Context(0, prec, 1 << 31, seed=SEED)
    n = 3
    ph = synth.centred_sphere(n, 0.3)
    dC = Q.qtt_from_phase_field(ctx, ph, n, (1.0, 10.0), (0.3, 0.25), None, 1e-10)
    p = Q.solve_params(1e-30, 6, 1e-10, 32)
    C1, i1, _ = Q.ls_solve_ceff(ctx, dC, p)
    ctx.set_concurrency(6)
    C6, i6, _ = Q.ls_solve_ceff(ctx, dC, p)
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert np.abs(C6 - C1).max() <= tol * np.abs(C1).max()
    ctx.close()


def test_fp32_products_of_rank_one_fields(Q):
    """FP32 mode with a truncation threshold below single precision: the
    products of rank-1 strain fields keep only real directions (columns at
    the rounding-noise floor of the SVD count as zero). Before that, noise
    directions were kept with non-orthogonal vectors and the SFFT product of
    a unit strain came out wrong by a factor ~3."""
    n = 3
    lam0 = dense.reference_lame((1.0, 20.0), (0.3, 0.3))
    ops = {"sfft": oq.sfft_operator(n, 1e-12), "gamma": oq.gamma_qtt(n, *lam0, 1e-8)}
    ctx = Q.Context(0, Q.QTT_FP32, 1 << 30, seed=SEED)
    try:
        for name, op in ops.items():
            cores, diag = to_lib_op(op)
            top = ctx.op(cores, diag)
            for k in (0, 3):
                x = oq.e_tt(n, np.eye(6)[k])
                y, rc = Q.qtt_op_apply(ctx, top, ctx.tt(x), 1e-12, 32, 16, apply_id=3)
                ref = oq.tto_full(op) @ oq.tt_full(x).reshape(-1)
                assert rel(oq.tt_full(y.cores()).reshape(-1), ref) < 1e-5, (name, k)
    finally:
        ctx.close()


def test_fp32_laminate_solve(Q):
    """A laminate (broadcast x1, x2) is solved exactly in two iterations in
    exact arithmetic; FP32 mode at eps_tt 1e-8 (below single precision)
    converges the same way and matches the dense oracle."""
    n = 3
    phb = synth.laminate(n, 2)
    E, nu = (1.0, 20.0), (0.3, 0.3)
    ctx = Q.Context(0, Q.QTT_FP32, 1 << 30, seed=SEED)
    try:
        dC = Q.qtt_from_phase_field(ctx, phb, n, E, nu, None, 1e-8)
        C, infos, rc = Q.ls_solve_ceff(ctx, dC, Q.solve_params(1e-5, 30, 1e-8, 32), loads=[0, 1, 3])
        Cd, imag, its = dense.ceff(synth.broadcast_dense(phb, n), E, nu, tol=1e-10, loads=[0, 1, 3])
        assert all(i["iters"] <= 4 for i in infos)
        for k in (0, 1, 3):
            assert np.abs(C[:, k] - Cd[:, k]).max() < 1e-5 * np.abs(Cd).max()
    finally:
        ctx.close()


def test_tf32x3_contractions_vs_oracle(Q):
    """Split-TF32 tensor-core contractions (FP32 context, TF32X3 mode): exact
    products (sketch rank above the product rank) of the Green and SFFT
    operators against the dense oracle product, at FP32-level accuracy: the
    hi*hi products and the hi*lo + lo*hi corrections are accumulated apart
    (one shared accumulator lost the corrections' low bits: 2.3e-5)."""
    n = 3
    rng = np.random.default_rng(21)
    ops = {"gamma": oq.gamma_qtt(n, 2.0, 1.0, 1e-12), "sfft": oq.sfft_operator(n)}
    x = random_tt(rng, qtt_dims(n), [1] + [min(6 * 2 ** k, 2 ** (3 * n - k), 9) for k in range(3 * n)] + [1])
    x, _ = oq.tt_round(x, 1e-14, 1000)
    ctx = Q.Context(0, Q.QTT_FP32, 1 << 30, seed=SEED)
    try:
        ctx.set_contraction(Q.QTT_CONTRACT_TF32X3)
        for name, op in ops.items():
            cores, diag = to_lib_op(op)
            y, rc = Q.qtt_op_apply(ctx, ctx.op(cores, diag), ctx.tt(x), 1e-12, 200, 16, apply_id=5)
            exact = oq.tto_full(op) @ oq.tt_full(x).reshape(-1)
            assert rel(oq.tt_full(y.cores()).reshape(-1), exact) < 1e-5, name
    finally:
        ctx.close()
    c64 = Q.Context(0, Q.QTT_FP64, 1 << 28, seed=SEED)
    try:
        with pytest.raises(Q.QttError):
            c64.set_contraction(Q.QTT_CONTRACT_TF32X3)
    finally:
        c64.close()


def test_tf32x3_mode_eight_spheres_16(Q):
    """The 16^3 8-sphere case in FP32 mode with split-TF32 tensor-core
    contractions meets the same 1e-4 C_eff goal as the SIMT contractions."""
    w = synth.spheres256(n=4)
    ctx = Q.Context(0, Q.QTT_FP32, 4 << 30, seed=SEED)
    try:
        ctx.set_contraction(Q.QTT_CONTRACT_TF32X3)
        dC = Q.qtt_from_phase_field(ctx, w.phase, w.n, w.E, w.nu, None, w.eps_tt, w.rmax)
        C, infos, rc = Q.ls_solve_ceff(ctx, dC, Q.solve_params(w.tol, 80, w.eps_tt, w.rmax),
                                       loads=[0])
        Cd, imag, its = dense.ceff(w.phase, w.E, w.nu, tol=1e-8, loads=[0])
        assert infos[0]["iters"] < 40 and infos[0]["residual"] < w.tol
        assert np.abs(C[:, 0] - Cd[:, 0]).max() < 1e-4 * np.abs(Cd).max()
    finally:
        ctx.close()


@pytest.mark.parametrize("mode", ["TF32X3", "TC"])
def test_tensor_core_contractions_n4_vs_oracle(Q, mode):
    """Split-TF32 contractions on the tensor cores (mma.sync kernel, or the
    tcgen05/TMA/TMEM kernel for the unbatched products of at least 64 x 32 x
    64) in a product large enough to use them: the Green operator at n = 4
    (13 cores) times a TT of ranks up to 40, against the oracle's exact
    product (Table 2), at FP32-level accuracy: within 3x the error of the same
    product with FP32 SIMT contractions (the FP32 sketching and factorisations
    set that level: 2.3e-5 measured for the split-TF32 mma.sync path)."""
    n = 4
    rng = np.random.default_rng(31)
    G = oq.gamma_qtt(n, 2.0, 1.0, 1e-12)
    dims = qtt_dims(n)
    L = len(dims)
    ranks = [1] + [min(6 * 2 ** k, 2 ** (L - 1 - k), 40) for k in range(L - 1)] + [1]
    x = random_tt(rng, dims, ranks)
    exact = oq.tt_full(oq.tto_apply_exact(G, x)).reshape(-1)
    cores, diag = to_lib_op(G)
    ctx = Q.Context(0, Q.QTT_FP32, 4 << 30, seed=SEED)
    try:
        y, rc = Q.qtt_op_apply(ctx, ctx.op(cores, diag), ctx.tt(x), 1e-12, 1000, 16, apply_id=3)
        e_simt = rel(y.to_dense().reshape(-1), exact)
        ctx.set_contraction(getattr(Q, f"QTT_CONTRACT_{mode}"))
        ctx.set_profiling(True)
        ctx.profile(reset=True)
        y, rc = Q.qtt_op_apply(ctx, ctx.op(cores, diag), ctx.tt(x), 1e-12, 1000, 16, apply_id=3)
        ctx.profile()
        if mode == "TC":
            assert ctx.last_tc_launches > 0
        e_tc = rel(y.to_dense().reshape(-1), exact)
        assert e_simt < 1e-4 and e_tc < 3 * e_simt + 1e-6, (e_tc, e_simt)
    finally:
        ctx.close()


def test_contraction_kernels_accuracy(Q):
    """Each contraction kernel on a random complex 512 x 256 x 1024 product
    against an FP64 GEMM of the same FP32 operands, within the FP32
    accumulation bound 4 sqrt(K') u (K' = 2048 real terms, u = 2^-24, i.e.
    1.1e-5). Measured: SIMT 2.9e-7, split-TF32 mma.sync 6.4e-7 (within 3x
    SIMT, also asserted), tcgen05 4.8e-6: its tensor-core accumulation keeps
    fewer low bits per addition than the SIMT FMA chain."""
    ctx = Q.Context(0, Q.QTT_FP32, 1 << 30, seed=SEED)
    try:
        err = {}
        for mode in ("SIMT", "TF32X3", "TC"):
            ms, e = Q.qtt_contraction_bench(ctx, getattr(Q, f"QTT_CONTRACT_{mode}"), 512, 256,
                                            1024, 3)
            assert ms > 0
            err[mode] = e
        bound = 4.0 * (2 * 1024) ** 0.5 * 2.0 ** -24
        assert max(err.values()) < bound, err
        assert err["TF32X3"] < 3 * err["SIMT"] + 1e-7, err
    finally:
        ctx.close()


def test_gamma_operator_centered_vs_oracle(Q, ctx64):
    """The Centered-scheme Green TTO (App. A table, k = i sin q) built on the
    device from the monomials of s/|s|, against the oracle's TT-SVD of its
    Centered Green field, for two reference media."""
    n = 3
    for lam0, mu0 in [(3.5, 1.25), (0.7, 4.0)]:
        op = Q.qtt_gamma_operator(ctx64, n, lam0, mu0, Q.QTT_SCHEME_CENTERED, 1e-12)
        G = oq.tto_full(from_lib_op(op.cores(), op.shape()[3]))
        ref = oq.tto_full(oq.gamma_qtt(n, lam0, mu0, 1e-12, scheme="centered"))
        assert rel(G, ref) < 1e-9
        direct = oq.tto_full(oq.gamma_qtt(n, lam0, mu0, 1e-12))
        assert rel(G, direct) > 1e-3


def test_ls_solve_centered_vs_dense_oracle(Q, ctx64):
    """The full solve with the Centered scheme against the dense FFT scheme
    with the same Green operator (Alg. 1), 8^3 sphere, loads e11 and e23."""
    n = 3
    ph = synth.centred_sphere(n, 0.3)
    E, nu = (1.0, 10.0), (0.3, 0.3)
    dC = Q.qtt_from_phase_field(ctx64, ph, n, E, nu, None, 1e-10)
    p = Q.solve_params(1e-6, 500, 1e-9, 64, Q.QTT_SCHEME_CENTERED)
    C, infos, rc = Q.ls_solve_ceff(ctx64, dC, p, loads=[0, 3])
    Cd, imag, its = dense.ceff(ph, E, nu, tol=1e-6, loads=[0, 3], scheme="centered")
    for k in (0, 3):
        assert np.abs(C[:, k] - Cd[:, k]).max() < 1e-5 * np.abs(Cd).max()


def test_rank_estimate_two_orders(Q, ctx64):
    """Applicability estimate (Sec. 5.2): the stiffness-TTO rank of a laminate
    does not grow with the order; a sphere's does. The rank at the lower
    order is the oracle's TT-SVD rank of the same field (within one, the
    device truncating the reduced k-row field)."""
    E, nu = (1.0, 10.0), (0.3, 0.3)
    lam0 = dense.reference_lame(E, nu)
    lam = Q.qtt_rank_estimate(ctx64, synth.laminate(5, 8), synth.laminate(6, 8), 5, E, nu, 1e-8,
                              n_target=11)
    assert abs(lam["growth"] - 1.0) < 1e-12 and lam["rank_target"] == lam["rank_n"]
    sph = Q.qtt_rank_estimate(ctx64, synth.centred_sphere(3, 0.3), synth.centred_sphere(4, 0.3), 3,
                              E, nu, 1e-8, n_target=8)
    assert sph["growth"] > 1.5
    ref = max(oq.tt_ranks(oq.stiffness_qtt(synth.centred_sphere(3, 0.3), 3, E, nu, lam0, 1e-8)))
    assert abs(sph["rank_n"] - ref) <= 1
