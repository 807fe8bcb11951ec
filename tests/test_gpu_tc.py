"""The trailing update of the two-stage reduction (A22 -= Y Z^H + Z Y^H) on the
tensor cores (split-bfloat16 products, float32 accumulation) and on the FP32
pipe, through the C ABI, against the same update in float64 on the host; and
the whole eigen-solve with either update against LAPACK."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs(batch, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((batch, n, n)) + 1j * rng.standard_normal((batch, n, n))
    A = (A + np.conj(np.swapaxes(A, 1, 2))) / 2
    Y = rng.standard_normal((batch, 16, n)) + 1j * rng.standard_normal((batch, 16, n))
    Z = 0.3 * (rng.standard_normal((batch, 16, n)) + 1j * rng.standard_normal((batch, 16, n)))
    return A, Y, Z


def _reference(A, Y, Z):
    # columns of Y and Z are the 16 panel vectors: U V^H with U = Y^T (n x 16)
    Yt = np.swapaxes(Y, 1, 2)
    Zt = np.swapaxes(Z, 1, 2)
    return A - Yt @ np.conj(np.swapaxes(Zt, 1, 2)) - Zt @ np.conj(np.swapaxes(Yt, 1, 2))


# float32 rounding of the inputs alone moves the result by ~2^-24 of the
# largest term; the products add their own error (measured on GB300 at n = 256:
# 3e-8, 1.5e-7 and 7e-7 of the largest term for tc = 0, 6 and 3).
TOL = {0: 2e-6, 6: 2e-6, 3: 1e-4}


@pytest.mark.parametrize("tc", [0, 6, 3])
@pytest.mark.parametrize("n,batch", [(38, 1), (300, 2), (514, 1)])
def test_her2k_matches_float64(tc, n, batch):
    import paper_1611_09784_gb300 as pkg
    A, Y, Z = _inputs(batch, n, 7 + n)
    got = pkg.her2k(A, Y, Z, tc_products=tc)
    ref = _reference(A, Y, Z)
    scale = np.max(np.abs(A)) + 32 * np.max(np.abs(Y)) * np.max(np.abs(Z))
    err = np.max(np.abs(got - ref)) / scale
    assert err < TOL[tc], f"tc={tc} n={n}: relative error {err:.3e}"


def test_her2k_six_products_are_float32_class():
    # Six split products drop only terms below ~3 * 2^-24 relative; what
    # remains is the tensor cores' own float32 accumulation (a few ulp of the
    # partial sums), within an order of magnitude of the FP32 pipe's error and
    # below the three-product form, which adds the bfloat16 rounding of the
    # low part.
    import paper_1611_09784_gb300 as pkg
    A, Y, Z = _inputs(2, 256, 3)
    ref = _reference(A, Y, Z)
    e6 = np.max(np.abs(pkg.her2k(A, Y, Z, tc_products=6) - ref))
    e3 = np.max(np.abs(pkg.her2k(A, Y, Z, tc_products=3) - ref))
    e0 = np.max(np.abs(pkg.her2k(A, Y, Z, tc_products=0) - ref))
    assert e6 <= 10 * e0 + 1e-12, (e6, e0)
    assert 2 * e6 <= e3, (e6, e3)


def test_her2k_leaves_rows_and_columns_of_zero_operands_unchanged():
    import paper_1611_09784_gb300 as pkg
    A, Y, Z = _inputs(1, 200, 11)
    Y[:, :, 150:] = 0
    Z[:, :, 150:] = 0
    got = pkg.her2k(A, Y, Z, tc_products=6)
    assert np.array_equal(got[:, 150:, 150:], A[:, 150:, 150:].astype(np.complex64).astype(np.complex128))


@pytest.mark.parametrize("tc", [0, 6, 3])
@pytest.mark.parametrize("n", [162, 600])
def test_eigvalsh_with_either_trailing_update(tc, n):
    import paper_1611_09784_gb300 as pkg
    rng = np.random.default_rng(n)
    H = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    H = (H + H.conj().T) / 2
    got = pkg.eigvalsh(H, precision="fp32", refine64_iters=1, tc_products=tc)[0]
    ref = np.linalg.eigvalsh(H)
    norm = np.max(np.abs(ref))
    tol = (2e-5 if tc != 3 else 5e-4) * norm
    assert np.max(np.abs(np.sort(got) - ref)) < tol


def test_her2k_tensor_cores_need_even_dimension():
    import paper_1611_09784_gb300 as pkg
    A, Y, Z = _inputs(1, 37, 1)
    with pytest.raises(pkg.IdosError):
        pkg.her2k(A, Y, Z, tc_products=6)
    got = pkg.her2k(A, Y, Z, tc_products=0)   # the FP32 pipe takes any dimension
    assert np.max(np.abs(got - _reference(A, Y, Z))) < 1e-4


def test_fp32_tensor_path_against_fp64_path_full_size_graphene():
    """The large-level comparison of the float32 path (tensor-core trailing
    update) with the float64-only GPU path, at N = 32 (n = 2048), one sample:
    eigenvalues within 1e-4 eV and IDoS within 1e-5."""
    import paper_1611_09784_gb300 as pkg
    from synthetic import workload
    w = workload("graphene_stress")
    out = {}
    for prec in ("fp32", "fp64"):
        cfg = dict(w["model"], p=w["p"], levels=[(32, 1)], e_min=w["e_min"], e_max=w["e_max"], n_E=w["n_E"],
                   delta=w["delta"], smoothing=w["smoothing"], precision=prec, refine64_iters=1, tc_products=6)
        m = pkg.create_model(cfg)
        out[prec] = m.eval_idos(32, 1, None, w["seed"], 0, 3, want_eigs=True)
        m.close()
    (q32, e32), (q64, e64) = out["fp32"], out["fp64"]
    keep = ~np.isnan(e64[0])
    assert np.array_equal(keep, ~np.isnan(e32[0]))
    assert np.max(np.abs(np.sort(e32[0][keep]) - np.sort(e64[0][keep]))) < 1e-4
    assert np.max(np.abs(q32 - q64)) < 1e-5


def _w_case(n, batch, k, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((batch, n, n)) + 1j * rng.standard_normal((batch, n, n))
    A = (A + np.conj(np.swapaxes(A, 1, 2))) / 2
    YT = rng.standard_normal((batch, 16, n)) + 1j * rng.standard_normal((batch, 16, n))
    m = n - k - 16
    A22 = A[:, k + 16:, k + 16:]
    V = np.swapaxes(YT[:, :, :m], 1, 2)           # (batch, m, 16)
    ref = np.zeros_like(YT)
    ref[:, :, :m] = np.swapaxes(A22 @ V, 1, 2)
    # per entry, sum_x |A22[r][x]| |V[x][c]|: the scale of a dot product's
    # rounding error
    bound = np.ones(YT.shape)
    bound[:, :, :m] = np.swapaxes(np.abs(A22) @ np.abs(V), 1, 2)
    return A, YT, ref, bound, m


@pytest.mark.parametrize("mode", [2, 1, 0])
@pytest.mark.parametrize("n,batch,k", [(48, 1, 0), (300, 2, 16), (514, 1, 0), (1030, 2, 496), (2048, 1, 0)])
def test_stage1_w_matches_float64(mode, n, batch, k):
    # W = A22 (Y T): the tensor-core kernel (six split-bfloat16 products,
    # float32 accumulation, the hi*hi and the smaller products in separate
    # accumulators) and the FP32-pipe kernels against float64.  Each entry's
    # error is measured against sum |A22| |V|: rounding the inputs to float32
    # alone gives about 2^-24 of it, the float32 sums a few more units.
    import paper_1611_09784_gb300 as pkg
    A, YT, ref, bound, m = _w_case(n, batch, k, 100 + n + k)
    got = pkg.stage1_w(A, YT, k=k, mode=mode)
    assert np.all(got[:, :, m:] == 0)
    err = np.max(np.abs(got - ref) / bound)
    assert err < 5e-7, f"mode={mode} n={n} k={k}: error {err:.3e} of sum |A22| |V|"


def test_stage1_w_tensor_cores_track_fp32_pipe():
    # the tensor-core W is float32-class: within a small factor of the FP32
    # pipe's own error against float64
    import paper_1611_09784_gb300 as pkg
    A, YT, ref, bound, m = _w_case(640, 2, 32, 5)
    e2 = np.max(np.abs(pkg.stage1_w(A, YT, k=32, mode=2) - ref) / bound)
    e1 = np.max(np.abs(pkg.stage1_w(A, YT, k=32, mode=1) - ref) / bound)
    assert e2 <= 8 * e1 + 1e-9, (e2, e1)
