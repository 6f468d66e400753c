"""Single cases of the library's kernels on seeded displaced icospheres, sized for a profiler capture.

    python -m paper_2203_12339_gb300.profile_case --nu 48 --K 12 --J 16 --precision bf16
    python -m paper_2203_12339_gb300.profile_case --case relight_frame --nu 128 --K 16 --J 25 --amp 0.15 \
        --octaves 5 --seed 2 --keep 0.05 --copies 13
    python -m paper_2203_12339_gb300.profile_case --case relight_batch --meshes 256 --edits 1024

The basis is fitted on the device from the seeded PCA materials (n_r = 1024, r_max = 40 mm,
eta = 1.3, Section 3.2), the scene is the icosphere of the benchmark recipe with 10 nu^2 + 2
vertices.  Every step runs through the C-ABI library; nothing here computes on the host.
"""
import argparse

import numpy as np
import torch

from . import scene, tsr


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--nu", type=int, default=48)
    ap.add_argument("--K", type=int, default=12)
    ap.add_argument("--J", type=int, default=16)
    ap.add_argument("--amp", type=float, default=0.1)
    ap.add_argument("--octaves", type=int, default=3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--precision", default="bf16", help="comma-separated list of bf16, bf16x3, fp32")
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--case", default="transfer", choices=["transfer", "relight_frame", "relight_batch"])
    ap.add_argument("--keep", type=float, default=0.05, help="relight_frame: kept fraction of the Haar coefficients")
    ap.add_argument("--copies", type=int, default=13, help="relight_frame: compressed copies, one RGB edit each")
    ap.add_argument("--meshes", type=int, default=256, help="relight_batch: meshes of the uneven batch")
    ap.add_argument("--edits", type=int, default=1024, help="relight_batch: material edits relit on every mesh")
    a = ap.parse_args(argv)
    if a.case == "relight_batch":
        relight_batch(a)
        return
    sa, ss = scene.pca_materials(256, seed=0)
    basis, _ = tsr.fit_pca_basis(torch.tensor(sa, device="cuda"), torch.tensor(ss, device="cuda"), 1.3, 1024, 40.0,
                                 a.K)
    sc = scene.make_scene(a.nu, K=a.K, J=a.J, amp=a.amp, octaves=a.octaves, seed=a.seed)
    pos = torch.tensor(np.ascontiguousarray(sc.mesh.pos.astype(np.float32).T), device="cuda")
    area = torch.tensor(sc.mesh.area.astype(np.float32), device="cuda")
    T = torch.tensor(sc.T.astype(np.float32), device="cuda")
    if a.case == "transfer":
        for prec in a.precision.split(","):
            for _ in range(a.repeat):
                tsr.precompute_transfer(basis, pos, area, T, prec)
    else:
        # the relight frame: `copies` compressed transfers (distinct buffers), one RGB edit each, relit by one call
        M = tsr.precompute_transfer(basis, pos, area, T, "bf16")
        copies = [tsr.haar_compress(M, a.nu, a.keep) for _ in range(a.copies)]
        del M
        esa, ess, eeta = scene.edit_materials(a.copies, seed=8)
        _, g32, _ = tsr.project_material(basis, torch.tensor(esa, device="cuda"), torch.tensor(ess, device="cuda"),
                                         torch.tensor(eeta, device="cuda"))
        light = torch.tensor(sc.light.astype(np.float32), device="cuda")
        g_frame = g32.reshape(a.copies, 1, 3, a.K).contiguous()
        for _ in range(a.repeat):
            tsr.relight_many(copies, g_frame, light)
    torch.cuda.synchronize()
    tsr.stream_status()
    print(f"ok: case={a.case} N={sc.n} K={a.K} J={a.J} precision={a.precision}")


def relight_batch(a):
    """The uneven batch (meshes of 642-40,962 vertices, seeds 1000 + b, amplitude 0.1, 3 octaves), K = 12,
    J = 16: BF16 transfer of all meshes in one call, Step 2 of every mesh (top 10 %), then three relights of
    `edits` shared material edits on every mesh in one tsr_relight_many call each."""
    K, J = 12, 16
    nus = scene.batched_nus(a.meshes, seed=4)
    meshes = [scene.make_scene(int(nu), K=K, J=J, amp=0.1, octaves=3, seed=1000 + b) for b, nu in enumerate(nus)]
    offs = np.concatenate([[0], np.cumsum([m.n for m in meshes])]).astype(np.int64)
    pos = torch.tensor(np.concatenate([m.mesh.pos for m in meshes]).astype(np.float32).T.copy(), device="cuda")
    area = torch.tensor(np.concatenate([m.mesh.area for m in meshes]).astype(np.float32), device="cuda")
    T = torch.tensor(np.concatenate([m.T for m in meshes], axis=1).astype(np.float32), device="cuda")
    light = torch.tensor(meshes[0].light.astype(np.float32), device="cuda")
    sa, ss = scene.pca_materials(256, seed=0)
    basis, _ = tsr.fit_pca_basis(torch.tensor(sa, device="cuda"), torch.tensor(ss, device="cuda"), 1.3, 1024, 40.0, K)
    esa, ess, eeta = scene.edit_materials(a.edits, seed=6)
    _, g32, _ = tsr.project_material(basis, torch.tensor(esa, device="cuda"), torch.tensor(ess, device="cuda"),
                                     torch.tensor(eeta, device="cuda"))
    g_all = g32.unsqueeze(0).expand(a.meshes, a.edits, 3, K).contiguous()
    M = tsr.precompute_transfer_batched(basis, offs, pos, area, T, "bf16")
    comps = tsr.haar_compress_batched(M, offs, 0.10)
    B = torch.empty(a.edits * 3 * int(offs[-1]), device="cuda")
    for _ in range(3):
        tsr.relight_many(comps, g_all, light, out=B)
    torch.cuda.synchronize()
    tsr.stream_status()
    print(f"ok: case=relight_batch meshes={a.meshes} vertices={int(offs[-1])} edits={a.edits}")


if __name__ == "__main__":
    main()
