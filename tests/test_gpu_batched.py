"""Batched transfer over meshes of uneven size: one persistent launch (BF16) or per-mesh launches (FP32),
against the oracle per mesh; the plan API, its autotuner and CUDA-graph capture; per-mesh compression of
the batched M in place and the relight of all meshes in one call."""
import numpy as np
import pytest

from oracle import tsr_oracle as O
from paper_2203_12339_gb300 import scene

pytestmark = pytest.mark.gpu
K, J = 12, 16
NUS = [8, 12, 9, 16, 10, 13, 8]   # 642 .. 2,562 vertices (the uneven-batch range starts at 642), ragged tiles


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_12339_gb300 import build
    build.build()
    from paper_2203_12339_gb300 import tsr
    sa, ss = scene.pca_materials(256, seed=0)
    f, _ = O.fit_pca_basis(sa, ss, 1.3, 1024, 40.0, K)
    meshes = [scene.make_scene(nu, K=K, J=J, amp=0.1, seed=10 + b) for b, nu in enumerate(NUS)]
    offs = np.concatenate([[0], np.cumsum([m.n for m in meshes])]).astype(np.int64)
    pos = np.concatenate([m.mesh.pos for m in meshes]).astype(np.float32)
    area = np.concatenate([m.mesh.area for m in meshes]).astype(np.float32)
    T = np.concatenate([m.T for m in meshes], axis=1).astype(np.float32)
    refs = [O.transfer_full(f, pos[offs[b]:offs[b + 1]], area[offs[b]:offs[b + 1]], T[:, offs[b]:offs[b + 1]])
            for b in range(len(meshes))]
    d = dict(pos=torch.tensor(pos.T.copy(), device="cuda"), area=torch.tensor(area, device="cuda"),
             T=torch.tensor(T, device="cuda"))
    return torch, tsr, tsr.basis_create(f), offs, d, refs


def _check(M, offs, refs, tol):
    for b, ref in enumerate(refs):
        got = M[:, :, offs[b]:offs[b + 1]]
        err = np.linalg.norm((got - ref).reshape(K, -1), axis=1) / np.linalg.norm(ref.reshape(K, -1), axis=1)
        assert err.max() <= tol, (b, err.max())


@pytest.mark.parametrize("precision,tol", [("bf16", 2e-3), ("fp32", 1e-5)])
def test_batched_matches_oracle_per_mesh(env, precision, tol):
    torch, tsr, basis, offs, d, refs = env
    M = tsr.precompute_transfer_batched(basis, offs, d["pos"], d["area"], d["T"], precision)
    tsr.stream_status()
    _check(M.cpu().numpy(), offs, refs, tol)


def test_plan_autotune_and_graph_capture(env):
    torch, tsr, basis, offs, d, refs = env
    plan = tsr.BatchPlan(basis, offs, J, "bf16")
    M = torch.zeros((K, J, int(offs[-1])), device="cuda")
    best = plan.autotune(d["pos"], d["area"], d["T"], out=M)
    info = plan.info()
    assert best > 0
    assert (info["generator"], info["param"]) in [("series", 1), ("series", 2), ("series", 3)] + [("table", kb) for kb in (4, 8, 12, 16)]
    assert info["units"] == sum((offs[b + 1] - offs[b] + 127) // 128 for b in range(len(NUS)))
    plan.run(d["pos"], d["area"], d["T"], out=M)           # warm (allocator pools, function attributes)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            plan.run(d["pos"], d["area"], d["T"], out=M)
    torch.cuda.current_stream().wait_stream(s)
    M.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    tsr.stream_status()
    _check(M.cpu().numpy(), offs, refs, 2e-3)


def test_batched_compress_recompress_and_relight(env):
    """Step 2 on the batched M read in place equals compressing each mesh's columns alone (bit-exact: same
    kernels on the same values); recompress refills the handles for a new M inside a CUDA graph; the relight
    of all meshes in one call (five edits: basis images + combine) equals the per-mesh relight within FP32
    reordering (2e-6)."""
    torch, tsr, basis, offs, d, refs = env
    M = tsr.precompute_transfer_batched(basis, offs, d["pos"], d["area"], d["T"], "fp32")
    comps = tsr.haar_compress_batched(M, offs, 0.1)
    for b, c in enumerate(comps):
        alone = tsr.haar_compress(M[:, :, offs[b]:offs[b + 1]].contiguous(), NUS[b], 0.1)
        for x, y in zip(c.export(), alone.export()):
            assert torch.equal(x, y), b
    M2 = M * 1.5 - 0.25 * M.flip(-1)
    torch.cuda.synchronize()
    tsr.haar_recompress_batched(M2, offs, comps)   # warm (scratch pools)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            tsr.haar_recompress_batched(M2, offs, comps)
    torch.cuda.current_stream().wait_stream(s)
    tsr.haar_recompress_batched(M, offs, comps)    # back to M, then the graph refills from M2
    g.replay()
    torch.cuda.synchronize()
    for b, c in enumerate(comps):
        alone = tsr.haar_compress(M2[:, :, offs[b]:offs[b + 1]].contiguous(), NUS[b], 0.1)
        for x, y in zip(c.export(), alone.export()):
            assert torch.equal(x, y), b
    rng = np.random.default_rng(12)
    E = 5
    gg = torch.tensor(rng.standard_normal((len(NUS), E, 3, K)).astype(np.float32), device="cuda")
    light = torch.tensor(rng.standard_normal(J).astype(np.float32), device="cuda")
    Bs = tsr.relight_many(comps, gg, light)
    for b, c in enumerate(comps):
        want = tsr.relight(c, gg[b], light)
        err = ((Bs[b] - want).reshape(E * 3, -1).norm(dim=1) / want.reshape(E * 3, -1).norm(dim=1)).max().item()
        assert err <= 2e-6, (b, err)
    tsr.stream_status()
