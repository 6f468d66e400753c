"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (per-k normwise over the compared rows for M, per (edit, channel)
normwise for B, relative for the rest):
  transfer FP32 <= 1e-5, split BF16 <= 1e-4, BF16 <= 2e-3;
  Haar, relight and its adjoint (FP32 arithmetic on identical inputs) <= 2e-6;
  FP64 basis / projection <= the Jacobi-vs-LAPACK perturbation bound below.
"""
import math

import numpy as np
import pytest

from oracle import tsr_oracle as O
from paper_2203_12339_gb300 import scene

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16x3": 1e-4, "bf16": 2e-3}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_12339_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def tsr(torch_cuda):
    from paper_2203_12339_gb300 import tsr as T
    return T


@pytest.fixture(scope="module")
def oracle_basis16():
    sa, ss = scene.pca_materials(256, seed=0)
    return O.fit_pca_basis(sa, ss, 1.3, 1024, 40.0, 16)


def _dev(torch, a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _normwise_k(got, ref):
    """max over k of ||dM[k]||_F / ||M[k]||_F."""
    d = np.linalg.norm((got - ref).reshape(got.shape[0], -1), axis=1)
    n = np.linalg.norm(ref.reshape(ref.shape[0], -1), axis=1)
    return float(np.max(d / n))


def _elementwise_k(got, ref):
    """max over k of max|dM[k]| / max|M[k]| (reading R31's element-wise figure): a localised
    error on a few rows, which the normwise figure dilutes over all rows, shows here."""
    d = np.abs(got - ref).reshape(got.shape[0], -1).max(axis=1)
    n = np.abs(ref).reshape(ref.shape[0], -1).max(axis=1)
    return float(np.max(d / n))


def _check_M(got, ref, precision):
    nw, ew = _normwise_k(got, ref), _elementwise_k(got, ref)
    assert nw <= TOL[precision], ("normwise", nw)
    assert ew <= TOL[precision], ("elementwise", ew)
    return nw, ew


# ------------------------------------------------------------------ Section 2.2
def test_fit_pca_basis_matches_oracle(torch_cuda, tsr, oracle_basis16):
    torch = torch_cuda
    f_ref, s_ref = oracle_basis16
    sa, ss = scene.pca_materials(256, seed=0)
    basis, sv = tsr.fit_pca_basis(_dev(torch, sa), _dev(torch, ss), 1.3, 1024, 40.0, 16)
    f = basis.table().cpu().numpy()
    sv = sv.cpu().numpy()
    assert sv.shape == (256,)
    # singular values: both SVDs are backward stable, |ds_k| <~ c eps s_0
    assert np.all(np.abs(sv[:16] - s_ref[:16]) <= 1e-13 * s_ref[0] + 1e-11 * s_ref[:16])
    # singular vectors: perturbation bound eps * s_0 / gap_k
    for k in range(16):
        gap = min(s_ref[k - 1] - s_ref[k] if k > 0 else np.inf, s_ref[k] - s_ref[k + 1])
        tol = 2e-13 * s_ref[0] / gap + 1e-13
        assert np.max(np.abs(f[k] - f_ref[k])) <= tol, (k, np.max(np.abs(f[k] - f_ref[k])), tol)
    assert np.max(np.abs(f @ f.T - np.eye(16))) < 1e-12


def test_fit_pca_basis_odd_material_count(torch_cuda, tsr):
    torch = torch_cuda
    sa, ss = scene.pca_materials(37, seed=9)
    f_ref, s_ref = O.fit_pca_basis(sa, ss, 1.2, 200, 30.0, 5)
    basis, sv = tsr.fit_pca_basis(_dev(torch, sa), _dev(torch, ss), 1.2, 200, 30.0, 5)
    assert np.max(np.abs(basis.table().cpu().numpy() - f_ref)) < 1e-9
    assert np.allclose(sv.cpu().numpy()[:5], s_ref[:5], rtol=1e-11)


def test_project_material_and_jacobian(torch_cuda, tsr, oracle_basis16):
    torch = torch_cuda
    f_ref, _ = oracle_basis16
    basis = tsr.basis_create(f_ref)
    sa, ss, eta = scene.edit_materials(50, seed=5)
    g, g32, dg = tsr.project_material(basis, _dev(torch, sa), _dev(torch, ss), _dev(torch, eta), jacobian=True)
    g_ref = O.project_material(f_ref, sa, ss, eta)
    assert np.max(np.abs(g.cpu().numpy() - g_ref)) <= 1e-12 * np.max(np.abs(g_ref))
    assert np.array_equal(g32.cpu().numpy(), g.cpu().numpy().astype(np.float32))
    r = O.radius_grid()
    d_a, d_s, d_e = O.dipole_rd_partials(r[None, None, :], sa[..., None], ss[..., None], eta[:, None, None])
    jac_ref = np.stack([d_a @ f_ref.T, d_s @ f_ref.T, d_e @ f_ref.T], axis=-1)
    dgc = dg.cpu().numpy()
    for q in range(3):
        scale = np.max(np.abs(jac_ref[..., q]))
        assert np.max(np.abs(dgc[..., q] - jac_ref[..., q])) <= 1e-11 * scale


def test_project_material_backward(torch_cuda, tsr, oracle_basis16):
    torch = torch_cuda
    f_ref, _ = oracle_basis16
    basis = tsr.basis_create(f_ref[:12])
    sa, ss, eta = scene.edit_materials(7, seed=8)
    dLdg = np.random.default_rng(0).standard_normal((7, 3, 12)).astype(np.float32)
    dsa, dss, de = tsr.project_material_backward(basis, _dev(torch, sa), _dev(torch, ss), _dev(torch, eta),
                                                 _dev(torch, dLdg))
    ra, rs, re = O.project_material_vjp(f_ref[:12], sa, ss, eta, dLdg.astype(np.float64))
    for got, ref in ((dsa, ra), (dss, rs), (de, re)):
        got = got.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref))


# ------------------------------------------------------------------ Eq. 6-7 transfer
def _scene_arrays(nu, K, J, amp, seed):
    """The scene's arrays; J beyond the 25 coefficients of four SH bands (the library takes up to 32)
    repeats the first transport rows, so every row keeps the statistics of real transport."""
    sc = scene.make_scene(nu, K=K, J=min(J, 25), amp=amp, seed=seed)
    T = sc.T.astype(np.float32)
    if J > 25:
        T = np.concatenate([T, T[:J - 25]])
    return sc, sc.mesh.pos.astype(np.float32), sc.mesh.area.astype(np.float32), T


@pytest.mark.parametrize("precision", ["fp32", "bf16", "bf16x3"])
@pytest.mark.parametrize("nu,K,J", [(9, 8, 9), (16, 12, 16), (5, 16, 25), (3, 3, 4)])
def test_transfer_full_small(torch_cuda, tsr, oracle_basis16, precision, nu, K, J):
    """Whole M on meshes that span several 128-row tiles with a ragged tail (812, 2562, 252, 92 vertices)."""
    torch = torch_cuda
    f_ref, _ = oracle_basis16
    sc, pos, area, T = _scene_arrays(nu, K, J, 0.12, 3)
    basis = tsr.basis_create(f_ref[:K])
    M = tsr.precompute_transfer(basis, _dev(torch, pos.T), _dev(torch, area), _dev(torch, T), precision)
    tsr.stream_status()
    M_ref = O.transfer_full(f_ref[:K], pos, area, T)
    _check_M(M.cpu().numpy(), M_ref, precision)


@pytest.mark.parametrize("nu,K,J,seed", [(1, 8, 9, 0), (2, 8, 9, 3), (4, 8, 9, 1), (4, 16, 25, 2), (4, 16, 32, 6),
                                         (6, 12, 16, 3), (7, 12, 16, 4), (8, 12, 16, 5)])
def test_transfer_bf16_coarse_meshes(torch_cuda, tsr, oracle_basis16, nu, K, J, seed):
    """BF16 on coarse meshes (12 to 642 vertices), where a few close pairs carry much of M: the
    near pairs (r < max(r_max / 16, 2h)) are summed exactly in FP32, so the bound holds with margin;
    J = 32 takes the widest records, accumulators and near-field staging."""
    torch = torch_cuda
    f_ref, _ = oracle_basis16
    sc, pos, area, T = _scene_arrays(nu, K, J, 0.1 if nu > 1 else 0.0, seed)
    basis = tsr.basis_create(f_ref[:K])
    M = tsr.precompute_transfer(basis, _dev(torch, pos.T), _dev(torch, area), _dev(torch, T), "bf16")
    tsr.stream_status()
    M_ref = O.transfer_full(f_ref[:K], pos, area, T)
    nw, ew = _check_M(M.cpu().numpy(), M_ref, "bf16")
    assert nw <= 1e-3, nw   # the normwise gate (R31) with a 2x margin; element-wise within 2e-3 above


def test_transfer_bf16_generators_and_series_fallback(torch_cuda, tsr, oracle_basis16, monkeypatch):
    """The two BF16 far-field generators (the 12-term series and the table) each meet the bound on
    the same mesh; a basis the series cannot represent (a step at 10 mm) is rejected by the
    series check at creation and the transfer takes the table, still within the bound."""
    torch = torch_cuda
    f_ref, _ = oracle_basis16
    sc, pos, area, T = _scene_arrays(20, 12, 16, 0.1, 3)
    args = (_dev(torch, pos.T), _dev(torch, area), _dev(torch, T))
    basis = tsr.basis_create(f_ref[:12])
    err, used = basis.far_series()
    assert used and err < 1e-3, err
    M_ref = O.transfer_full(f_ref[:12], pos, area, T)
    M_series = tsr.precompute_transfer(basis, *args, "bf16").cpu().numpy()
    monkeypatch.setenv("TSR_BF16_GENERATOR", "table")
    M_table = tsr.precompute_transfer(basis, *args, "bf16").cpu().numpy()
    monkeypatch.delenv("TSR_BF16_GENERATOR")
    tsr.stream_status()
    _check_M(M_series, M_ref, "bf16")
    _check_M(M_table, M_ref, "bf16")
    r = O.radius_grid()
    f_step = f_ref[:4].copy()
    f_step[:, r > 10.0] *= 0.5
    b_step = tsr.basis_create(f_step)
    err, used = b_step.far_series()
    assert not used and err > 2e-3, err
    M = tsr.precompute_transfer(b_step, *args, "bf16")
    tsr.stream_status()
    _check_M(M.cpu().numpy(), O.transfer_full(f_step, pos, area, T), "bf16")


@pytest.mark.parametrize("K,J", [(12, 16), (16, 25)])
def test_transfer_series_generator_layouts(torch_cuda, tsr, oracle_basis16, monkeypatch, K, J):
    """Every layout of the far-field series generator on a 4,002-vertex mesh: one group of 16 warps,
    two or three groups of 8 warps; the A operand in tensor memory, in shared memory, or split
    between them (the first terms of a slot in tensor memory).  They form the same BF16 products and
    issue the same MMAs in the same order, so M is bit-identical across them, and within the BF16
    bound of the oracle."""
    torch = torch_cuda
    f_ref, _ = oracle_basis16
    sc, pos, area, T = _scene_arrays(20, K, J, 0.1, 3)
    args = (_dev(torch, pos.T), _dev(torch, area), _dev(torch, T))
    basis = tsr.basis_create(f_ref[:K])
    assert basis.far_series()[1]
    # (groups, A in shared memory, hybrid)
    layouts = [("1", "0", "0"), ("2", "0", "0"), ("3", "0", "0"), ("2", "1", "0"), ("3", "1", "0")] if J <= 16 else \
              [("1", "0", "0"), ("2", "1", "0"), ("3", "1", "0"), ("2", "1", "1"), ("3", "1", "1")]
    out = {}
    for conc, smem, hyb in layouts:
        monkeypatch.setenv("TSR_CHEB_CONC", conc)
        monkeypatch.setenv("TSR_CHEB_SMEM", smem)
        monkeypatch.setenv("TSR_CHEB_HYB", hyb)
        out[(conc, smem, hyb)] = tsr.precompute_transfer(basis, *args, "bf16").cpu().numpy()
    tsr.stream_status()
    first = out[layouts[0]]
    for key, M in out.items():
        assert np.array_equal(M, first), key
    _check_M(first, O.transfer_full(f_ref[:K], pos, area, T), "bf16")


@pytest.mark.parametrize("K,J", [(12, 16), (16, 25)])
def test_transfer_streamk_cut_tiles(torch_cuda, tsr, oracle_basis16, K, J):
    """4,002 vertices = 32 tiles x 251 steps over ~125 equal stage ranges: most tiles are cut into
    pieces that the fix-up sums (the last, 34-row tile too).
    - split BF16 and BF16 against the oracle (1e-4, 2e-3 with a 2x margin: on this mesh basis 1
      has ~10x cancellation in M, which a plain BF16 contraction of every pair, self pair
      excepted, turned into a 3.7e-3 error);
    - BF16 against the same mesh through the batched path, whose units are whole tiles (same BF16
      products, other accumulation segments; the tensor-core accumulation truncates, ~1e-7 per step
      relative to the running sum): 2e-4, where a lost or doubled piece would be off by >1e-2;
    - two runs bit-identical (the fix-up adds the pieces in a fixed order)."""
    torch = torch_cuda
    f_ref, _ = oracle_basis16
    sc, pos, area, T = _scene_arrays(20, K, J, 0.1, 3)
    assert sc.n == 4002
    basis = tsr.basis_create(f_ref[:K])
    args = (_dev(torch, pos.T), _dev(torch, area), _dev(torch, T))
    M_ref = O.transfer_full(f_ref[:K], pos, area, T)
    Ms = tsr.precompute_transfer(basis, *args, "bf16x3")
    _check_M(Ms.cpu().numpy(), M_ref, "bf16x3")
    M1 = tsr.precompute_transfer(basis, *args, "bf16")
    nw, ew = _check_M(M1.cpu().numpy(), M_ref, "bf16")
    assert nw <= 1e-3, nw
    M2 = tsr.precompute_transfer(basis, *args, "bf16")
    Mb = tsr.precompute_transfer_batched(basis, [0, sc.n], *args, "bf16")
    tsr.stream_status()
    assert torch.equal(M1, M2)
    d = (M1 - Mb).reshape(K, -1).norm(dim=1) / Mb.reshape(K, -1).norm(dim=1)
    assert float(d.max()) <= 2e-4, d


def test_transfer_tiny_mesh_and_single_basis(torch_cuda, tsr, oracle_basis16):
    torch = torch_cuda
    f_ref, _ = oracle_basis16
    sc, pos, area, T = _scene_arrays(1, 1, 1, 0.0, 0)   # 12 vertices, K = J = 1
    basis = tsr.basis_create(f_ref[:1])
    M_ref = O.transfer_full(f_ref[:1], pos, area, T)
    for precision in ("fp32", "bf16", "bf16x3"):
        M = tsr.precompute_transfer(basis, _dev(torch, pos.T), _dev(torch, area), _dev(torch, T), precision)
        tsr.stream_status()
        _check_M(M.cpu().numpy(), M_ref, precision)


@pytest.mark.parametrize("precision", ["fp32", "bf16", "bf16x3"])
def test_transfer_full_size_sampled_rows(torch_cuda, tsr, oracle_basis16, precision):
    """40,962-vertex displaced sphere, K=12, J=16 (the benchmark workload): 1,024 sampled output rows."""
    torch = torch_cuda
    f_ref, _ = oracle_basis16
    w = scene.WORKLOADS["disp40962_k12_j16"]
    sc, pos, area, T = _scene_arrays(w["nu"], w["K"], w["J"], w["amp"], w["seed"])
    basis = tsr.basis_create(f_ref[:12])
    M = tsr.precompute_transfer(basis, _dev(torch, pos.T), _dev(torch, area), _dev(torch, T), precision)
    tsr.stream_status()
    rows = scene.sample_rows(sc.n, 1024, seed=7)
    M_ref = O.transfer_rows(f_ref[:12], pos, area, T, rows)
    _check_M(M.cpu().numpy()[:, :, rows], M_ref, precision)


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
def test_transfer_largest_sampled_rows(torch_cuda, tsr, oracle_basis16, precision):
    """163,842-vertex displaced sphere, K=16, J=25: 128 sampled output rows."""
    torch = torch_cuda
    f_ref, _ = oracle_basis16
    w = scene.WORKLOADS["disp163842_k16_j25"]
    sc, pos, area, T = _scene_arrays(w["nu"], w["K"], w["J"], w["amp"], w["seed"])
    basis = tsr.basis_create(f_ref)
    M = tsr.precompute_transfer(basis, _dev(torch, pos.T), _dev(torch, area), _dev(torch, T), precision)
    tsr.stream_status()
    rows = scene.sample_rows(sc.n, 128, seed=7)
    M_ref = O.transfer_rows(f_ref, pos, area, T, rows)
    _check_M(M.cpu().numpy()[:, :, rows], M_ref, precision)


# ------------------------------------------------------------------ Eq. 9-10 Haar
@pytest.mark.parametrize("nu", [1, 3, 4, 5, 16, 33, 64, 100, 128])
def test_haar_forward_inverse(torch_cuda, tsr, nu):
    torch = torch_cuda
    rng = np.random.default_rng(nu)
    X = rng.standard_normal((7, 10 * nu * nu + 2)).astype(np.float32)
    Xw = tsr.haar_forward(_dev(torch, X), nu).cpu().numpy()
    ref = O.chart_to_wavelet(X, nu)
    assert np.max(np.abs(Xw - ref)) <= 2e-6 * np.max(np.abs(ref))
    back = tsr.haar_inverse(_dev(torch, ref.astype(np.float32)), nu).cpu().numpy()
    assert np.max(np.abs(back - X)) <= 2e-6 * np.max(np.abs(X))


@pytest.mark.parametrize("nu", [1, 2, 3, 5, 8, 16, 33, 64, 128])
def test_cdf97_forward_inverse(torch_cuda, tsr, nu):
    """The paper's Step-2 wavelet (CDF 9/7): analysis and synthesis against the oracle's lifting."""
    torch = torch_cuda
    rng = np.random.default_rng(200 + nu)
    X = rng.standard_normal((5, 10 * nu * nu + 2)).astype(np.float32)
    Xw = tsr.cdf97_forward(_dev(torch, X), nu).cpu().numpy()
    ref = O.chart_to_cdf97(X, nu)
    assert np.max(np.abs(Xw - ref)) <= 2e-6 * np.max(np.abs(ref))
    back = tsr.cdf97_inverse(_dev(torch, ref.astype(np.float32)), nu).cpu().numpy()
    assert np.max(np.abs(back - X)) <= 2e-6 * np.max(np.abs(X))


@pytest.mark.parametrize("nu", [1, 2, 3, 4, 6, 8])
def test_cdf97_inverse_transpose_matches_the_matrix(torch_cuda, tsr, nu):
    """S^T (the reverse mode of the relight) against the transpose of the oracle's explicit synthesis matrix."""
    torch = torch_cuda
    rng = np.random.default_rng(300 + nu)
    dB = rng.standard_normal((4, 10 * nu * nu + 2)).astype(np.float32)
    got = tsr.cdf97_inverse_transpose(_dev(torch, dB), nu).cpu().numpy()
    want = dB.astype(np.float64) @ O.cdf97_synthesis_matrix(nu)
    assert np.max(np.abs(got - want)) <= 2e-6 * np.max(np.abs(want))


@pytest.mark.parametrize("nu", [16, 64, 128])
def test_cdf97_adjoint_identity(torch_cuda, tsr, nu):
    """<S c, y> = <c, S^T y> between the GPU synthesis and its transpose (sizes the explicit matrix cannot reach)."""
    torch = torch_cuda
    rng = np.random.default_rng(400 + nu)
    P = O.chart_side(nu)
    c = rng.standard_normal((3, 10 * P * P + 2)).astype(np.float32)
    y = rng.standard_normal((3, 10 * nu * nu + 2)).astype(np.float32)
    Sc = tsr.cdf97_inverse(_dev(torch, c), nu).cpu().numpy().astype(np.float64)
    STy = tsr.cdf97_inverse_transpose(_dev(torch, y), nu).cpu().numpy().astype(np.float64)
    lhs = np.sum(Sc * y, axis=1)
    rhs = np.sum(c * STy, axis=1)
    scale = np.sqrt(np.sum(Sc ** 2, axis=1) * np.sum(y ** 2, axis=1))
    assert np.max(np.abs(lhs - rhs) / scale) <= 1e-6


def test_cdf97_compress_relight_and_adjoint(torch_cuda, tsr):
    """Step 2 with CDF 9/7 (top fraction and energy rules): kept sets equal the oracle's on the GPU's
    own coefficients; relight and its adjoint against the oracle in the same wavelet."""
    torch = torch_cuda
    nu, K, J, E = 8, 5, 9, 3
    N = 10 * nu * nu + 2
    rng = np.random.default_rng(31)
    M = (rng.standard_normal((K, J, N)) * np.exp(-np.arange(N) % 64 / 16.0)).astype(np.float32)
    Md = _dev(torch, M)
    Mw = tsr.cdf97_forward(Md.reshape(K * J, N), nu).reshape(K, J, -1).cpu().numpy()
    n_rows = Mw.shape[-1]
    g = rng.standard_normal((E, 3, K)).astype(np.float32)
    light = rng.standard_normal(J).astype(np.float32)
    dB = rng.standard_normal((E, 3, N)).astype(np.float32)
    for rule, param, want in (("top", 0.1, O.select_top(Mw, nu, 0.1)), ("energy", 0.97, O.select_energy(Mw, nu, 0.97))):
        comp = tsr.compress(Md, nu, "cdf97", rule, param)
        row_ptr, col, _ = (t.cpu().numpy() for t in comp.export())
        got = _mask_from_csr(row_ptr, col, n_rows, K * J).reshape(K, J, n_rows)
        assert np.array_equal(got, want), rule
        kept = np.where(got, Mw.astype(np.float64), 0.0)
        B = tsr.relight(comp, _dev(torch, g), _dev(torch, light)).cpu().numpy()
        B_ref = O.relight(kept, nu, g.astype(np.float64), light.astype(np.float64), wavelet="cdf97")
        assert np.max(np.abs(B - B_ref)) <= 1e-5 * np.max(np.abs(B_ref))
        B1 = tsr.relight(comp, _dev(torch, g[:1]), _dev(torch, light)).cpu().numpy()   # direct path (3 vectors)
        assert np.max(np.abs(B1 - B_ref[:1])) <= 1e-5 * np.max(np.abs(B_ref[:1]))
        dg, dl = tsr.relight_backward(comp, _dev(torch, g), _dev(torch, light), _dev(torch, dB))
        dg_ref, dl_ref = O.relight_vjp(kept, nu, g.astype(np.float64), light.astype(np.float64),
                                       dB.astype(np.float64), wavelet="cdf97")
        assert np.max(np.abs(dg.cpu().numpy() - dg_ref)) <= 1e-5 * np.max(np.abs(dg_ref))
        assert np.max(np.abs(dl.cpu().numpy() - dl_ref)) <= 1e-5 * np.max(np.abs(dl_ref))


# ------------------------------------------------------------------ Step 2 selection (bit-exact)
def _mask_from_csr(row_ptr, col, n_rows, KJ):
    mask = np.zeros((KJ, n_rows), dtype=bool)
    for w in range(n_rows):
        for q in range(row_ptr[w], row_ptr[w + 1]):
            mask[col[q], w] = True
    return mask


@pytest.mark.parametrize("nu,p", [(4, 0.1), (3, 0.37), (8, 0.05), (2, 1.0)])
def test_select_and_pack_exact(torch_cuda, tsr, nu, p):
    torch = torch_cuda
    K, J = 3, 5
    P = O.chart_side(nu)
    rng = np.random.default_rng(nu)
    Mw = (rng.integers(-20, 21, size=(K, J, 10 * P * P + 2)) * 0.25).astype(np.float32)   # many exact ties
    comp = tsr.wavelet_compress(_dev(torch, Mw), nu, p)
    row_ptr, col, val = (t.cpu().numpy() for t in comp.export())
    n_rows = 10 * P * P + 2
    assert comp.nnz == K * J * (O.keep_count(p, 10 * P * P) + 2)
    assert row_ptr[0] == 0 and row_ptr[-1] == comp.nnz
    for w in range(n_rows):
        assert np.all(np.diff(col[row_ptr[w]:row_ptr[w + 1]]) > 0)
    got = _mask_from_csr(row_ptr, col, n_rows, K * J).reshape(K, J, n_rows)
    want = O.select_top(Mw, nu, p)
    assert np.array_equal(got, want)
    # values are the kept coefficients, bit for bit
    for w in range(0, n_rows, 7):
        for q in range(row_ptr[w], row_ptr[w + 1]):
            assert val[q] == Mw.reshape(K * J, n_rows)[col[q], w]


@pytest.mark.parametrize("data", ["spread", "zeros"])
def test_select_large_rows_exact(torch_cuda, tsr, data):
    """Rows of 40,960 chart coefficients (nu = 40: 64 x 64 charts) take the block selection: a 12-bit
    first digit over the row, then the gathered keys of that digit in shared memory (values spread over
    many binades) or more digits over the row (90 % exact zeros and eighths: more than 4,096 equal keys
    and ties everywhere).  Bit-exact against the oracle's top-p mask (ties by lower index)."""
    torch = torch_cuda
    nu, K, J, p = 40, 2, 3, 0.1
    P = O.chart_side(nu)
    n_rows = 10 * P * P + 2
    rng = np.random.default_rng(7)
    if data == "spread":
        Mw = rng.standard_normal((K, J, n_rows)) * np.exp(rng.uniform(-12.0, 3.0, (K, J, n_rows)))
    else:
        Mw = np.where(rng.random((K, J, n_rows)) < 0.9, 0.0, np.round(rng.standard_normal((K, J, n_rows)) * 8) / 8)
    Mw = Mw.astype(np.float32)
    comp = tsr.wavelet_compress(_dev(torch, Mw), nu, p)
    row_ptr, col, val = (t.cpu().numpy() for t in comp.export())
    got = _mask_from_csr(row_ptr, col, n_rows, K * J).reshape(K, J, n_rows)
    assert np.array_equal(got, O.select_top(Mw, nu, p))


def _energy_boundary_ok(row, e, n_gpu):
    """True if n_gpu reaches the energy threshold and n_gpu - 1 does not, both within FP64
    rounding of the summation order (the two sides add the same exact squares in different orders)."""
    c = np.asarray(row, dtype=np.float64)
    order = np.lexsort((np.arange(c.size), -np.abs(c)))
    cum = np.cumsum(c[order] ** 2)
    total, tol = cum[-1], 1e-12 * cum[-1]
    return cum[n_gpu - 1] >= e * total - tol and (n_gpu == 1 or cum[n_gpu - 2] < e * total + tol)


@pytest.mark.parametrize("nu,e", [(4, 0.95), (8, 0.9), (16, 0.98), (33, 0.95), (64, 0.99)])
def test_energy_select_and_pack(torch_cuda, tsr, nu, e):
    """Energy rule (Section 3, precompute Step 2): per (k, j) the kept set equals the oracle's on the
    same FP32 wavelet coefficients (the GPU's own Haar output), columns of varying length."""
    torch = torch_cuda
    K, J = 3, 4
    P = O.chart_side(nu)
    n_coef = 10 * P * P
    rng = np.random.default_rng(100 + nu)
    N = 10 * nu * nu + 2
    decay = np.exp(-np.arange(N) % max(1, nu * nu) / max(1.0, nu * nu / 6.0))
    M = (rng.standard_normal((K, J, N)) * decay).astype(np.float32)
    Md = _dev(torch, M)
    Mw = tsr.haar_forward(Md.reshape(K * J, N), nu).reshape(K, J, -1).cpu().numpy()
    comp = tsr.haar_compress_energy(Md, nu, e)
    row_ptr, col, val = (t.cpu().numpy() for t in comp.export())
    n_rows = n_coef + 2
    got = _mask_from_csr(row_ptr, col, n_rows, K * J).reshape(K, J, n_rows)
    want = O.select_energy(Mw, nu, e)
    assert got[:, :, n_coef:].all()
    for k in range(K):
        for j in range(J):
            if np.array_equal(got[k, j], want[k, j]):
                continue
            n_gpu = int(got[k, j, :n_coef].sum())   # boundary decided within FP64 rounding: the set
            assert _energy_boundary_ok(Mw[k, j, :n_coef], e, n_gpu)   # must still be a prefix of the ranking
            order = np.lexsort((np.arange(n_coef), -np.abs(Mw[k, j, :n_coef]).astype(np.float64)))
            assert set(np.nonzero(got[k, j, :n_coef])[0].tolist()) == set(order[:n_gpu].tolist())
    assert comp.nnz == int(got.sum())
    for w in range(0, n_rows, 5):
        for q in range(row_ptr[w], row_ptr[w + 1]):
            assert val[q] == Mw.reshape(K * J, n_rows)[col[q], w]
    with pytest.raises(tsr.TsrError):
        tsr.haar_compress(Md, nu, 0.1, out=comp)   # data-dependent sizes: no recompression in place


def test_energy_rule_relight_and_adjoint(torch_cuda, tsr):
    """Relight and its adjoint through a handle with columns of different lengths (the adjoint
    walks the per-column lists by their offsets)."""
    torch = torch_cuda
    nu, K, J, E, e = 8, 6, 9, 4, 0.95
    N = 10 * nu * nu + 2
    rng = np.random.default_rng(21)
    M = (rng.standard_normal((K, J, N)) * np.exp(-np.arange(N) % 64 / 12.0)).astype(np.float32)
    Md = _dev(torch, M)
    Mw = tsr.haar_forward(Md.reshape(K * J, N), nu).reshape(K, J, -1).cpu().numpy()
    comp = tsr.haar_compress_energy(Md, nu, e)
    row_ptr, col, _ = (t.cpu().numpy() for t in comp.export())
    mask = _mask_from_csr(row_ptr, col, Mw.shape[-1], K * J).reshape(Mw.shape)
    counts = mask.sum(axis=-1)
    assert counts.min() < counts.max()            # the columns really differ in length
    kept = np.where(mask, Mw.astype(np.float64), 0.0)
    g = rng.standard_normal((E, 3, K)).astype(np.float32)
    light = rng.standard_normal(J).astype(np.float32)
    B = tsr.relight(comp, _dev(torch, g), _dev(torch, light)).cpu().numpy()
    B_ref = O.relight(kept, nu, g.astype(np.float64), light.astype(np.float64))
    assert np.max(np.abs(B - B_ref)) <= 1e-5 * np.max(np.abs(B_ref))
    dB = rng.standard_normal((E, 3, N)).astype(np.float32)
    dg, dl = tsr.relight_backward(comp, _dev(torch, g), _dev(torch, light), _dev(torch, dB))
    dg_ref, dl_ref = O.relight_vjp(kept, nu, g.astype(np.float64), light.astype(np.float64), dB.astype(np.float64))
    assert np.max(np.abs(dg.cpu().numpy() - dg_ref)) <= 1e-5 * np.max(np.abs(dg_ref))
    assert np.max(np.abs(dl.cpu().numpy() - dl_ref)) <= 1e-5 * np.max(np.abs(dl_ref))


# ------------------------------------------------------------------ Steps 3-5 relight
def _compressed_case(torch, tsr, nu, K, J, p, seed):
    rng = np.random.default_rng(seed)
    P = O.chart_side(nu)
    Mw = rng.standard_normal((K, J, 10 * P * P + 2)).astype(np.float32) * np.exp(-np.arange(10 * P * P + 2) % (P * P) / (P * P / 4.0)).astype(np.float32)
    comp = tsr.wavelet_compress(_dev(torch, Mw), nu, p)
    kept = np.where(O.select_top(Mw, nu, p), Mw.astype(np.float64), 0.0)
    return comp, kept


@pytest.mark.parametrize("nu,K,J,E,p", [(4, 8, 9, 5, 0.1), (5, 12, 16, 3, 0.2), (16, 16, 25, 2, 0.05), (1, 1, 1, 1, 1.0)])
def test_relight_matches_oracle(torch_cuda, tsr, nu, K, J, E, p):
    torch = torch_cuda
    comp, kept = _compressed_case(torch, tsr, nu, K, J, p, nu + K)
    rng = np.random.default_rng(1)
    g = rng.standard_normal((E, 3, K)).astype(np.float32)
    light = rng.standard_normal(J).astype(np.float32)
    B = tsr.relight(comp, _dev(torch, g), _dev(torch, light)).cpu().numpy()
    B_ref = O.relight(kept, nu, g.astype(np.float64), light.astype(np.float64))
    num = np.linalg.norm((B - B_ref).reshape(E * 3, -1), axis=1)
    den = np.linalg.norm(B_ref.reshape(E * 3, -1), axis=1)
    assert np.max(num / den) <= 2e-6


def _relight_err(B, B_ref):
    E = B_ref.shape[0]
    num = np.linalg.norm((B - B_ref).reshape(E * 3, -1), axis=1)
    den = np.linalg.norm(B_ref.reshape(E * 3, -1), axis=1)
    return float(np.max(num / den))


@pytest.mark.parametrize("nu,K,J,p", [(40, 3, 4, 0.1), (64, 2, 3, 0.05), (100, 2, 2, 0.05), (128, 2, 2, 0.05)])
def test_relight_one_edit_large_charts(torch_cuda, tsr, nu, K, J, p):
    """One and two edits on charts of 64^2 and 128^2 Morton positions (4 and 16 runs of 1,024 per chart;
    ragged nu = 40 and nu = 100 among them, up to the library's nu = 128): the fused product + inverse
    Haar per run against the oracle."""
    torch = torch_cuda
    comp, kept = _compressed_case(torch, tsr, nu, K, J, p, nu + 7)
    rng = np.random.default_rng(nu)
    light = rng.standard_normal(J).astype(np.float32)
    for E in (1, 2):
        g = rng.standard_normal((E, 3, K)).astype(np.float32)
        B = tsr.relight(comp, _dev(torch, g), _dev(torch, light)).cpu().numpy()
        B_ref = O.relight(kept, nu, g.astype(np.float64), light.astype(np.float64))
        assert _relight_err(B, B_ref) <= 2e-6, (E, _relight_err(B, B_ref))


@pytest.mark.parametrize("p", [1.0, 0.6])
def test_relight_dense_runs_many_windows(torch_cuda, tsr, p):
    """Every (p = 1) or most coefficients kept at K = 16, J = 25 on 64^2-position charts: a run's rows hold
    up to 1,023 x 400 entries, so the fused kernel's rows take up to 13 lane units each, span warp steps
    and cross the eight warp ranges, whose partial sums are chained.  One and two edits (3 and 6 vectors)
    and five edits (the 16 basis images + combine) against the oracle."""
    torch = torch_cuda
    nu, K, J = 64, 16, 25
    comp, kept = _compressed_case(torch, tsr, nu, K, J, p, 64)
    rng = np.random.default_rng(5)
    light = rng.standard_normal(J).astype(np.float32)
    for E in (1, 2, 5):
        g = rng.standard_normal((E, 3, K)).astype(np.float32)
        B = tsr.relight(comp, _dev(torch, g), _dev(torch, light)).cpu().numpy()
        B_ref = O.relight(kept, nu, g.astype(np.float64), light.astype(np.float64))
        assert _relight_err(B, B_ref) <= 2e-6, (E, _relight_err(B, B_ref))
        Bm = tsr.relight_many([comp], _dev(torch, g[None]), _dev(torch, light))[0].cpu().numpy()
        assert _relight_err(Bm, B_ref) <= 2e-6, (E, _relight_err(Bm, B_ref))


def test_relight_many_uneven_copies(torch_cuda, tsr):
    """tsr_relight_many over uneven copies (1 to 40 vertices per chart side, Haar and CDF 9/7): every
    copy against the oracle's relight of its own kept coefficients, for 1, 2 and 3 edits (fused launch,
    per-copy fallbacks); also more copies than one launch takes (32)."""
    torch = torch_cuda
    K, J = 4, 5
    nus = [1, 3, 5, 8, 16, 40, 17, 2]
    comps, kepts = [], []
    for i, nu in enumerate(nus):
        comp, kept = _compressed_case(torch, tsr, nu, K, J, 0.2, 100 + i)
        comps.append(comp)
        kepts.append(kept)
    # one CDF 9/7 copy (not fused: relit by tsr_relight inside the call)
    nu_c = 8
    N_c = 10 * nu_c * nu_c + 2
    rng = np.random.default_rng(5)
    Mc = (rng.standard_normal((K, J, N_c)) * np.exp(-np.arange(N_c) % 64 / 16.0)).astype(np.float32)
    Mcd = _dev(torch, Mc)
    Mcw = tsr.cdf97_forward(Mcd.reshape(K * J, N_c), nu_c).reshape(K, J, -1).cpu().numpy()
    comp_c = tsr.compress(Mcd, nu_c, "cdf97", "top", 0.2)
    comps.append(comp_c)
    kepts.append(np.where(O.select_top(Mcw, nu_c, 0.2), Mcw.astype(np.float64), 0.0))
    nus.append(nu_c)
    light = rng.standard_normal(J).astype(np.float32)
    for E in (1, 2, 3):
        g = rng.standard_normal((len(comps), E, 3, K)).astype(np.float32)
        Bs = tsr.relight_many(comps, _dev(torch, g), _dev(torch, light))
        torch.cuda.synchronize()
        for i, (B, kept, nu) in enumerate(zip(Bs, kepts, nus)):
            wav = "cdf97" if i == len(comps) - 1 else "haar"
            B_ref = O.relight(kept, nu, g[i].astype(np.float64), light.astype(np.float64), wavelet=wav)
            err = _relight_err(B.cpu().numpy(), B_ref)
            assert err <= (1e-5 if wav == "cdf97" else 2e-6), (E, i, nu, err)
    # 70 copies: three fused launches of at most 32 copies, results equal to relighting each alone
    many = [comps[i % 6] for i in range(70)]
    g = rng.standard_normal((70, 1, 3, K)).astype(np.float32)
    gd = _dev(torch, g)
    Bs = tsr.relight_many(many, gd, _dev(torch, light))
    for i in (0, 31, 32, 63, 64, 69):
        want = tsr.relight(many[i], gd[i], _dev(torch, light))
        assert torch.equal(Bs[i], want), i


@pytest.mark.parametrize("K,J,E", [(2, 3, 4), (5, 4, 7), (8, 9, 3), (16, 25, 5)])
def test_relight_many_factorised_batch(torch_cuda, tsr, K, J, E):
    """More than two edits: the light-contracted basis images of every copy in one fused pass (K of 2 to 16
    images per copy) and one combine over all copies and edits; copies of 1 to 16 runs per chart, ragged
    nu among them; every copy against the oracle."""
    torch = torch_cuda
    nus = [3, 8, 40, 100, 16]
    comps, kepts = [], []
    for i, nu in enumerate(nus):
        comp, kept = _compressed_case(torch, tsr, nu, K, J, 0.1, 200 + 7 * i + K)
        comps.append(comp)
        kepts.append(kept)
    rng = np.random.default_rng(K * J)
    light = rng.standard_normal(J).astype(np.float32)
    g = rng.standard_normal((len(comps), E, 3, K)).astype(np.float32)
    Bs = tsr.relight_many(comps, _dev(torch, g), _dev(torch, light))
    torch.cuda.synchronize()
    for i, (B, kept, nu) in enumerate(zip(Bs, kepts, nus)):
        B_ref = O.relight(kept, nu, g[i].astype(np.float64), light.astype(np.float64))
        err = _relight_err(B.cpu().numpy(), B_ref)
        assert err <= 2e-6, (i, nu, err)


def test_compressed_save_and_load_round_trip(torch_cuda, tsr, tmp_path):
    """Checkpoint/resume of a compressed transfer (top-fraction Haar, and energy-rule CDF 9/7): the loaded
    handle exports the same arrays and relights and back-propagates bit-identically."""
    torch = torch_cuda
    comp, _ = _compressed_case(torch, tsr, 20, 6, 9, 0.1, 77)
    nu_c, K, J = 8, 5, 9
    rng = np.random.default_rng(78)
    M = (rng.standard_normal((K, J, 10 * nu_c * nu_c + 2)) * np.exp(-np.arange(10 * nu_c * nu_c + 2) % 64 / 16.0))
    comp_c = tsr.compress(_dev(torch, M.astype(np.float32)), nu_c, "cdf97", "energy", 0.97)
    for i, c in enumerate((comp, comp_c)):
        path = str(tmp_path / f"c{i}.tsr")
        c.save(path)
        d = tsr.Compressed.load(path)
        assert (d.K, d.J, d.nu, d.nnz, d.n_rows) == (c.K, c.J, c.nu, c.nnz, c.n_rows)
        for x, y in zip(c.export(), d.export()):
            assert torch.equal(x, y)
        g = torch.tensor(rng.standard_normal((3, 3, c.K)).astype(np.float32), device="cuda")
        light = torch.tensor(rng.standard_normal(c.J).astype(np.float32), device="cuda")
        for E in (1, 3):
            assert torch.equal(tsr.relight(c, g[:E], light), tsr.relight(d, g[:E], light))
        dB = torch.randn((3, 3, c.n), device="cuda")
        for x, y in zip(tsr.relight_backward(c, g, light, dB), tsr.relight_backward(d, g, light, dB)):
            assert torch.equal(x, y)


def test_relight_many_rejects_mismatched_handles(torch_cuda, tsr):
    torch = torch_cuda
    a, _ = _compressed_case(torch, tsr, 4, 4, 5, 0.2, 1)
    b, _ = _compressed_case(torch, tsr, 4, 3, 5, 0.2, 2)
    g = torch.zeros((2, 1, 3, 4), device="cuda")
    with pytest.raises(tsr.TsrError):
        tsr.relight_many([a, b], g, torch.zeros(5, device="cuda"))


@pytest.mark.parametrize("nu,K,J,E,p", [(4, 8, 9, 5, 0.1), (5, 12, 16, 3, 0.2), (8, 16, 25, 11, 0.05)])
def test_relight_backward_matches_oracle(torch_cuda, tsr, nu, K, J, E, p):
    torch = torch_cuda
    comp, kept = _compressed_case(torch, tsr, nu, K, J, p, 3 * nu + K)
    rng = np.random.default_rng(2)
    g = rng.standard_normal((E, 3, K)).astype(np.float32)
    light = rng.standard_normal(J).astype(np.float32)
    dB = rng.standard_normal((E, 3, 10 * nu * nu + 2)).astype(np.float32)
    dg, dl = tsr.relight_backward(comp, _dev(torch, g), _dev(torch, light), _dev(torch, dB))
    dg_ref, dl_ref = O.relight_vjp(kept, nu, g.astype(np.float64), light.astype(np.float64), dB.astype(np.float64))
    assert np.max(np.abs(dg.cpu().numpy() - dg_ref)) <= 1e-5 * np.max(np.abs(dg_ref))
    assert np.max(np.abs(dl.cpu().numpy() - dl_ref)) <= 1e-5 * np.max(np.abs(dl_ref))


# ------------------------------------------------------------------ whole path
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_end_to_end_sphere2562(torch_cuda, tsr, precision):
    """Undisplaced 2,562-vertex sphere, K=8, J=9, marble: fit -> project -> transfer -> compress -> relight."""
    torch = torch_cuda
    w = scene.WORKLOADS["sphere2562_k8_j9"]
    sc, pos, area, T = _scene_arrays(w["nu"], w["K"], w["J"], w["amp"], w["seed"])
    sa, ss = scene.pca_materials(256, seed=0)
    f_ref, _ = O.fit_pca_basis(sa, ss, 1.3, 1024, 40.0, 8)
    basis, _ = tsr.fit_pca_basis(_dev(torch, sa), _dev(torch, ss), 1.3, 1024, 40.0, 8)
    msa, mss, meta = scene.marble(1)
    _, g32, _ = tsr.project_material(basis, _dev(torch, msa), _dev(torch, mss), _dev(torch, meta))
    g_ref = O.project_material(f_ref, msa, mss, meta)
    M = tsr.precompute_transfer(basis, _dev(torch, pos.T), _dev(torch, area), _dev(torch, T), precision)
    comp = tsr.haar_compress(M, w["nu"], 1.0)   # keep everything: no selection ambiguity
    B = tsr.relight(comp, g32, _dev(torch, sc.light.astype(np.float32))).cpu().numpy()
    tsr.stream_status()
    M_ref = O.transfer_full(f_ref, pos, area, T)
    B_ref = O.relight(O.chart_to_wavelet(M_ref, w["nu"]), w["nu"], g_ref, sc.light)
    rel = np.linalg.norm((B - B_ref).reshape(3, -1), axis=1) / np.linalg.norm(B_ref.reshape(3, -1), axis=1)
    assert rel.max() <= TOL[precision]


# ------------------------------------------------------------------ boundary behaviour
def test_invalid_arguments_are_rejected(torch_cuda, tsr, oracle_basis16):
    torch = torch_cuda
    f_ref, _ = oracle_basis16
    basis = tsr.basis_create(f_ref[:4])
    pos = torch.zeros((3, 11), device="cuda")
    with pytest.raises(tsr.TsrError) as e:
        tsr.precompute_transfer(basis, pos, torch.zeros(11, device="cuda"), torch.zeros((4, 11), device="cuda"))
    assert e.value.status == -1
    with pytest.raises(tsr.TsrError) as e:
        tsr.haar_forward(torch.zeros((2, 10 * 129 * 129 + 2), device="cuda"), 129)
    assert e.value.status == -1
    with pytest.raises(tsr.TsrError):
        tsr.precompute_transfer(basis, torch.zeros((3, 42), device="cuda"), torch.zeros(42, device="cuda"),
                                torch.zeros((33, 42), device="cuda"))


# ------------------------------------------------------------------ Fresnel factors (Eq. 3, Eq. 6)
def test_fresnel_output_and_reverse_mode(torch_cuda, tsr):
    torch = torch_cuda
    rng = np.random.default_rng(41)
    E, N = 5, 1037
    B = rng.standard_normal((E, 3, N)).astype(np.float32)
    eta = rng.uniform(1.0, 1.8, E)
    cos_o = np.concatenate([rng.uniform(-1, 1, N - 3), [0.0, 1.0, 1e-7]]).astype(np.float32)
    Bo = tsr.fresnel_output(_dev(torch, B), torch.tensor(eta, device="cuda"), _dev(torch, cos_o)).cpu().numpy()
    ref = O.fresnel_output(B, eta, cos_o)
    assert np.max(np.abs(Bo - ref)) <= 2e-6 * np.max(np.abs(ref))
    dBout = rng.standard_normal((E, 3, N)).astype(np.float32)
    dB, deta = tsr.fresnel_output_backward(_dev(torch, B), torch.tensor(eta, device="cuda"), _dev(torch, cos_o),
                                           _dev(torch, dBout))
    dB_ref, deta_ref = O.fresnel_output_vjp(B, eta, cos_o, dBout)
    assert np.max(np.abs(dB.cpu().numpy() - dB_ref)) <= 2e-6 * np.max(np.abs(dB_ref))
    assert np.max(np.abs(deta.cpu().numpy() - deta_ref)) <= 1e-4 * np.max(np.abs(deta_ref))


@pytest.mark.parametrize("J,eta", [(9, 1.3), (16, 1.5), (25, 1.0), (1, 1.2)])
def test_sh_transfer_with_incident_fresnel(torch_cuda, tsr, J, eta):
    """T[j, i] = A_l(eta) Y_lm(n_i) (Funk-Hecke) on a displaced mesh's normals, against the oracle."""
    torch = torch_cuda
    mesh = scene.icosphere(8, 0.12, 3, 4)
    normals = mesh.normal.astype(np.float32)
    T = tsr.sh_transfer(_dev(torch, normals.T), J, eta).cpu().numpy()
    ref = O.sh_transfer_fresnel(normals.astype(np.float64), J, eta)
    assert np.max(np.abs(T - ref)) <= 2e-6 * np.max(np.abs(ref))
    if eta == 1.0:
        assert np.max(np.abs(T - scene.sh_transfer(normals.astype(np.float64), J))) <= 2e-6


def test_view_dependent_render_end_to_end(torch_cuda, tsr, oracle_basis16):
    """Eq. 6 with both Fresnel factors on 252 vertices: T with the incident F_t at the precompute's eta,
    FP32 transfer, keep-all Haar compression, relight of two edits, output factor for a view direction."""
    torch = torch_cuda
    f_ref, _ = oracle_basis16
    K, J, nu = 6, 9, 5
    mesh = scene.icosphere(nu, 0.1, 3, 5)
    pos, area, normals = (a.astype(np.float32) for a in (mesh.pos, mesh.area, mesh.normal))
    T_ref = O.sh_transfer_fresnel(normals.astype(np.float64), J, 1.3)
    T = tsr.sh_transfer(_dev(torch, normals.T), J, 1.3)
    basis = tsr.basis_create(f_ref[:K])
    M = tsr.precompute_transfer(basis, _dev(torch, pos.T), _dev(torch, area), T, "fp32")
    comp = tsr.haar_compress(M, nu, 1.0)
    sa, ss, eta = scene.edit_materials(2, seed=12)
    g = O.project_material(f_ref[:K], sa, ss, eta)
    light = scene.sh_light(J, 3)
    view = np.array([0.3, -0.4, 0.866])
    cos_o = (normals @ (view / np.linalg.norm(view))).astype(np.float32)
    B = tsr.relight(comp, _dev(torch, g.astype(np.float32)), _dev(torch, light.astype(np.float32)))
    Bo = tsr.fresnel_output(B, torch.tensor(eta, device="cuda"), _dev(torch, cos_o)).cpu().numpy()
    M_ref = O.transfer_full(f_ref[:K], pos, area, T_ref.astype(np.float32))
    B_ref = O.relight(O.chart_to_wavelet(M_ref, nu), nu, g, light)
    ref = O.fresnel_output(B_ref, eta, cos_o)
    err = np.linalg.norm((Bo - ref).reshape(-1, Bo.shape[-1]), axis=1) / np.linalg.norm(ref.reshape(-1, ref.shape[-1]), axis=1)
    assert err.max() <= 1e-5, err


# ------------------------------------------------------------------ ray-cast visibility in T
def _vis_compare(T_gpu, T_ref, S):
    """Equal up to FP32 accumulation, except at the few vertices where a grazing ray's hit decision sits
    on a rounding boundary (a sample then moves by pi/S |Y_j| <= pi/S)."""
    diff = np.abs(T_gpu - T_ref).max(axis=0)
    tight = diff <= 1e-5 * np.abs(T_ref).max()
    assert tight.mean() >= 0.99, (tight.mean(), diff.max())
    assert diff.max() <= 2.0 * math.pi / S * 0.8


@pytest.mark.parametrize("nu,amp,seed,J,S,eta", [(6, 0.2, 3, 9, 64, 0.0), (8, 0.15, 5, 16, 128, 1.3)])
def test_visibility_transfer_matches_oracle(torch_cuda, tsr, nu, amp, seed, J, S, eta):
    torch = torch_cuda
    mesh = scene.icosphere(nu, amp, 3, seed)
    pos, normals = mesh.pos.astype(np.float32), mesh.normal.astype(np.float32)
    T = tsr.visibility_transfer(_dev(torch, pos.T), _dev(torch, normals.T),
                                torch.tensor(mesh.tris.astype(np.int32), device="cuda"), J, S, eta).cpu().numpy()
    T_ref = O.visibility_transfer(pos, mesh.tris, normals, J, S, eta=(eta if eta > 0 else None))
    _vis_compare(T, T_ref, S)
    unshadowed = O.sh_transfer_fresnel(normals.astype(np.float64), J, eta) if eta > 0 else scene.sh_transfer(normals, J)
    assert (T[0] < 0.97 * unshadowed[0]).any()          # the displaced mesh does shadow itself


def test_visibility_transfer_convex_sphere_and_single_triangle(torch_cuda, tsr):
    torch = torch_cuda
    mesh = scene.icosphere(4, 0.0, 3, 0)
    pos, normals = mesh.pos.astype(np.float32), mesh.normal.astype(np.float32)
    T = tsr.visibility_transfer(_dev(torch, pos.T), _dev(torch, normals.T),
                                torch.tensor(mesh.tris.astype(np.int32), device="cuda"), 9, 512).cpu().numpy()
    assert np.abs(T - scene.sh_transfer(normals, 9)).max() < 5e-3   # nothing blocked: the cosine quadrature
    # one triangle above one point: every ray blocked (the single-leaf path)
    pos1 = np.array([[0.0, 0.0, 0.0], [-1e4, -1e4, 1.0], [1e4, -1e4, 1.0], [0.0, 1e4, 1.0]], dtype=np.float32)
    nrm1 = np.array([[0.0, 0.0, 1.0]] * 4, dtype=np.float32)
    T1 = tsr.visibility_transfer(_dev(torch, pos1.T), _dev(torch, nrm1.T),
                                 torch.tensor([[1, 2, 3]], dtype=torch.int32, device="cuda"), 4, 64).cpu().numpy()
    assert np.abs(T1[:, 0]).max() == 0.0
