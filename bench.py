"""Benchmark of the translucent-transfer hot path on the 163,842-vertex displaced sphere.

One step = the per-scene path of the method on the largest single-GPU workload
(163,842 vertices, K = 16 PCA terms, J = 25 SH terms, 5 % of the Haar coefficients kept):
  project 13 RGB material edits (Section 2.2, FP64)
  -> transfer M[k,j,o] = sum_i A_i f_k(r_oi) T[j,i] in BF16 on the tensor cores, the near
     field exactly in FP32 (Section 3, Eq. 6-7)
  -> spatial Haar + top-5 % keep rule per (k, j) (Section 3.2, Eq. 9-10)
  -> relight of the 13 edits: one 1920 x 1080-equivalent frame of vertex shading
     (13 x 163,842 = 2.13 M shaded vertices; Section 4, Steps 3-5)
  -> reverse mode of relight and projection for L = 0.5 ||B||^2.
The PCA basis (Eq. 5) is fitted once before timing (a one-time set-up, setup_ms).

metric: transfer G pair.K.J/s = N^2 K J / step time / 1e9 (whole job, all ranks).
Beside it, measured outside the timed steps and each with its error against the FP64
oracle: the transfer in BF16, split BF16 and FP32 at 163,842 and 40,962 vertices; the
1080p-equivalent frame from 13 compressed copies; the 256-mesh uneven batch; the step's
own relit frame and gradients.
Multi-GPU: every rank processes its own scene (independent problems, weak scaling);
the only collectives are the barrier and the max of the timings.

--impl reference times the FP64 CPU oracle on a bounded sample of output rows of
the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "disp163842_k16_j25"        # headline: the largest single-GPU configuration
SIDE_WORKLOAD = "disp40962_k12_j16"    # the 40,962-vertex configuration, measured beside it
N_EDITS = 13                           # one 1920 x 1080-equivalent frame of vertex shading
KEEP = 0.05
METRIC = "transfer G pair.K.J/s"
UNIT = "G pair.K.J/s"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _traffic_record(name: str):
    """DRAM bytes per transfer launch from a committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", name)
    src = os.path.join(ROOT, "paper_2203_12339_gb300", "csrc", "transfer.cu")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh)
    with open(src, "rb") as fh:
        sha = hashlib.sha256(fh.read()).hexdigest()
    if rec.get("source_sha256") != sha:
        return None
    return rec.get("traffic_bytes_per_launch")


def _scene(name: str, rank: int = 0):
    from paper_2203_12339_gb300 import scene
    w = scene.WORKLOADS[name]
    sc = scene.make_scene(w["nu"], K=w["K"], J=w["J"], amp=w["amp"], octaves=w["octaves"],
                          seed=w["seed"] + 100 * rank)
    return w, sc


def _m_errors(got, ref) -> dict:
    """Transfer errors on sampled rows (reading R31): max over k of the normwise and the
    element-wise relative error, got and ref (K, J, rows)."""
    K = ref.shape[0]
    d = np.linalg.norm((got - ref).reshape(K, -1), axis=1) / np.linalg.norm(ref.reshape(K, -1), axis=1)
    e = np.abs(got - ref).reshape(K, -1).max(axis=1) / np.abs(ref).reshape(K, -1).max(axis=1)
    return {"normwise": float(d.max()), "elementwise": float(e.max())}


def _rel(got, ref) -> float:
    """max over leading rows of ||got - ref|| / ||ref|| (per edit and channel for B)."""
    g = np.asarray(got, dtype=np.float64).reshape(-1, np.asarray(got).shape[-1])
    r = np.asarray(ref, dtype=np.float64).reshape(-1, np.asarray(ref).shape[-1])
    return float(np.max(np.linalg.norm(g - r, axis=1) / np.linalg.norm(r, axis=1)))


def _dense_kept(comp, K: int, J: int) -> np.ndarray:
    """The kept wavelet coefficients of a compressed transfer as a dense (K, J, rows) FP64 array."""
    row_ptr, col, val = (t.cpu().numpy() for t in comp.export())
    rows = np.repeat(np.arange(comp.n_rows), np.diff(row_ptr))
    out = np.zeros((K * J, comp.n_rows))
    out[col[:len(rows)], rows] = val[:len(rows)]
    return out.reshape(K, J, comp.n_rows)


def _timed(fn, reps: int = 1):
    """(ms per call by CUDA events on the current stream, tensor-core transfer kernel ms per launch or None)."""
    import torch
    from paper_2203_12339_gb300 import tsr
    fn()
    torch.cuda.synchronize()
    tsr.kernel_timing_read()
    tsr.kernel_timing(True)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    tsr.kernel_timing(False)
    kms, n = tsr.kernel_timing_read()
    return a.elapsed_time(b) / reps, (kms / n if n else None)


class OracleChecks:
    """Errors against the FP64 oracle, computed in the oracle leg after all GPU timing.

    GPU measurements register (target dict, key, kind, GPU result, reference builder); run()
    imports the oracle, builds each reference once (memoised by name) and writes the error
    into the target: kind "M" gives the normwise and element-wise transfer errors, "rel" the
    max per-row relative error, "rel_list" the same over lists of arrays."""

    def __init__(self):
        self.items = []
        self.refs = {}

    def add(self, target: dict, key: str, kind: str, got, ref_name: str, ref_fn):
        self.items.append((target, key, kind, got, ref_name, ref_fn))

    def run(self) -> float:
        from oracle import tsr_oracle as O
        t = time.perf_counter()
        for target, key, kind, got, ref_name, ref_fn in self.items:
            if ref_name not in self.refs:
                self.refs[ref_name] = ref_fn(O)
            ref = self.refs[ref_name]
            if kind == "M":
                target[key] = _m_errors(got, ref)
            elif kind == "rel_list":   # arrays of different widths: the max over the pairs
                target[key] = max(_rel(g, r) for g, r in zip(got, ref))
            else:
                target[key] = _rel(got, ref)
        self.refs.clear()
        return time.perf_counter() - t


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"tsr_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.remove(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def transfer_sweep(tsr, basis, d, N, K, J, rows, peaks, checks, ref_name, ref_fn,
                   precs=("bf16", "bf16x3", "fp32")) -> dict:
    """The transfer of one mesh in each precision, timed alone (CUDA events around the call; the
    tensor-core kernel by its own events), with its error on the sampled rows against the oracle
    (registered in `checks`; ref_fn(O) builds the oracle's rows)."""
    import torch
    M = torch.empty((K, J, N), dtype=torch.float32, device=d["pos"].device)
    units = float(N) * N * K * J
    out = {}
    for prec in precs:
        ms, kms = _timed(lambda: tsr.precompute_transfer(basis, d["pos"], d["area"], d["T"], prec, out=M))
        tsr.stream_status()
        r = {"ms": round(ms, 3), "g_pair_kj_per_s": round(units / (ms * 1e-3) / 1e9, 1)}
        checks.add(r, "error_vs_oracle", "M", M.cpu().numpy()[:, :, rows], ref_name, ref_fn)
        if kms is not None:
            tf = 2.0 * units / (kms * 1e-3) / 1e12
            peak = float(peaks.get("bf16_tflops", 1900.0))
            r["tensor_kernel"] = {"ms": round(kms, 3), "tflops": round(tf, 1), "peak": peak,
                                  "frac": round(tf / peak, 4), "peak_kind": "bf16 burst (kernel timed alone)"}
        out[prec] = r
    del M
    return out


def relight_frame_1080p(tsr, dev, peaks, basis, M, w, sc, checks) -> dict:
    """A 1920x1080-equivalent relight frame: 13 copies (distinct buffers, so S streams 13 times)
    of the 163,842-vertex compressed transfer (K=16, J=25, 5 % kept), one RGB material edit each
    (projected once, Step 3), relit (Steps 4-5) by one tsr_relight_many call replayed as a CUDA
    graph.  HBM roofline on the algorithmic bytes of a frame, 13 x (nnz x 6 B + N x 12 B).  Error:
    three copies' B against the oracle's dense relight of the same kept coefficients."""
    import torch
    from paper_2203_12339_gb300 import scene
    copies = [tsr.haar_compress(M, w["nu"], KEEP) for _ in range(13)]
    esa, ess, eeta = scene.edit_materials(13, seed=8)
    light = torch.tensor(sc.light.astype(np.float32), device=dev)
    _, g32, _ = tsr.project_material(basis, torch.tensor(esa, device=dev), torch.tensor(ess, device=dev),
                                     torch.tensor(eeta, device=dev))   # Step 3: once per edit, not per frame
    g_frame = g32.reshape(13, 1, 3, w["K"]).contiguous()   # one RGB edit per copy
    out = torch.empty(13 * 3 * sc.n, device=dev, dtype=torch.float32)

    def frame():
        return tsr.relight_many(copies, g_frame, light, out=out)

    frame()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side, capture_error_mode="thread_local"):
            frame()
    torch.cuda.current_stream().wait_stream(side)
    graph.replay()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    reps = 50
    a.record()
    for _ in range(reps):
        graph.replay()
    b.record()
    torch.cuda.synchronize()
    tsr.stream_status()
    ms = a.elapsed_time(b) / reps
    N = sc.n
    frame_bytes = 13.0 * (copies[0].nnz * 6 + N * 12)
    achieved = frame_bytes / (ms * 1e-3) / 1e9
    peak = float(peaks.get("hbm_gbs", 6800.0))
    Cw = _dense_kept(copies[0], w["K"], w["J"]).astype(np.float32)
    sel = [0, 6, 12]
    B = out.reshape(13, 3, N)[sel].cpu().numpy()
    g = g32.cpu().numpy().astype(np.float64)[sel]
    light_h = sc.light.astype(np.float32)
    del copies
    res = {"workload": "13 x disp163842_k16_j25 compressed (5 % kept), 1 RGB edit each, Steps 4-5 by one "
                       "tsr_relight_many call (CUDA graph replay)",
           "fps": round(1e3 / ms, 1), "ms_per_frame": round(ms, 4),
           "error_vs_oracle": {"note": "copies 0, 6, 12 against the oracle's dense relight of the same kept "
                                       "coefficients, per edit and channel"},
           "hbm_roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                            "frac": round(achieved / peak, 4), "bytes_per_frame": int(frame_bytes)}}
    checks.add(res["error_vs_oracle"], "relight_rel", "rel", B, "frame1080p",
               lambda O: np.stack([O.relight(Cw, w["nu"], g[q:q + 1], light_h)[0] for q in range(len(sel))]))
    return res


def batched_scene(tsr, dev, peaks, checks, n_mesh: int = 256, n_edit: int = 1024) -> dict:
    """The uneven batch: n_mesh displaced icospheres (vertex counts log-uniform in 642-40,962, seeds 1000 + b,
    amplitude 0.1, 3 octaves), K=12, J=16.  One pass = the BF16 transfer of every mesh in one persistent launch
    (autotuned plan), Step 2 of every mesh read in place from the batched M (top 10 %), and the relight of
    n_edit material edits (projected once, shared by the meshes) on every mesh: basis images of all meshes in
    one fused pass, then one combine writing n_edit x 3 x sum(N) outputs.  Timed per stage (CUDA events,
    eager) and as one CUDA-graph replay of the whole pass.  Errors: M on 32 sampled rows of the three largest
    and the three smallest meshes against the oracle, and B of two meshes (4 edits) against the oracle's
    relight of the same kept coefficients."""
    import torch
    from paper_2203_12339_gb300 import scene
    K, J = 12, 16
    nus = scene.batched_nus(n_mesh, seed=4)
    meshes = [scene.make_scene(int(nu), K=K, J=J, amp=0.1, octaves=3, seed=1000 + b) for b, nu in enumerate(nus)]
    offs = np.concatenate([[0], np.cumsum([m.n for m in meshes])]).astype(np.int64)
    total = int(offs[-1])
    pos_h = np.concatenate([m.mesh.pos for m in meshes]).astype(np.float32)
    area_h = np.concatenate([m.mesh.area for m in meshes]).astype(np.float32)
    T_h = np.concatenate([m.T for m in meshes], axis=1).astype(np.float32)
    pos = torch.tensor(pos_h.T.copy(), device=dev)
    area = torch.tensor(area_h, device=dev)
    T = torch.tensor(T_h, device=dev)
    light_h = meshes[0].light.astype(np.float32)
    light = torch.tensor(light_h, device=dev)
    del meshes
    sa_pca, ss_pca = scene.pca_materials(256, seed=0)
    basis, _ = tsr.fit_pca_basis(torch.tensor(sa_pca, device=dev), torch.tensor(ss_pca, device=dev), 1.3, 1024,
                                 40.0, K)
    esa, ess, eeta = scene.edit_materials(n_edit, seed=6)
    _, g32, _ = tsr.project_material(basis, torch.tensor(esa, device=dev), torch.tensor(ess, device=dev),
                                     torch.tensor(eeta, device=dev))
    g_all = g32.unsqueeze(0).expand(n_mesh, n_edit, 3, K).contiguous()
    plan = tsr.BatchPlan(basis, offs, J, "bf16")
    M = torch.empty((K, J, total), device=dev, dtype=torch.float32)
    plan.autotune(pos, area, T, out=M)
    plan.run(pos, area, T, out=M)
    comps = tsr.haar_compress_batched(M, offs, 0.10)
    B = torch.empty(n_edit * 3 * total, device=dev, dtype=torch.float32)
    stages = (lambda: plan.run(pos, area, T, out=M),
              lambda: tsr.haar_recompress_batched(M, offs, comps),
              lambda: tsr.relight_many(comps, g_all, light, out=B))
    for fn in stages:
        fn()
    torch.cuda.synchronize()
    ms = []
    for fn in stages:
        reps = []
        for _ in range(3):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            reps.append(a.elapsed_time(b))
        ms.append(statistics.median(reps))
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side, capture_error_mode="thread_local"):
            for fn in stages:
                fn()
    torch.cuda.current_stream().wait_stream(side)
    graph.replay()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(3):
        graph.replay()
    b.record()
    torch.cuda.synchronize()
    tsr.stream_status()
    graph_ms = a.elapsed_time(b) / 3
    n_per = offs[1:] - offs[:-1]
    # what the oracle leg compares (outside the timed region); only the compared rows leave the GPU
    order = np.argsort(n_per, kind="stable")
    picks = [int(i) for i in list(order[-3:]) + list(order[:3])]
    m_cases = []
    for b_ in picks:
        o0, o1 = int(offs[b_]), int(offs[b_ + 1])
        rows = scene.sample_rows(o1 - o0, 32, seed=b_)
        idx = torch.tensor(o0 + rows, device=dev, dtype=torch.long)
        m_cases.append((o0, o1, rows, M.index_select(2, idx).cpu().numpy()))
    g_h = g32.cpu().numpy().astype(np.float64)[:4]
    b_cases = []
    base = 0   # B holds the meshes' [n_edit][3][N_b] blocks back to back
    for b_ in range(n_mesh):
        nb = int(n_per[b_])
        if b_ in (picks[0], picks[-1]):
            b_cases.append((int(nus[b_]), _dense_kept(comps[b_], K, J).astype(np.float32),
                            B[base:base + 4 * 3 * nb].reshape(4, 3, nb).cpu().numpy()))
        base += n_edit * 3 * nb
    pairs = float(np.sum(n_per.astype(np.float64) ** 2))
    out_bytes = 4.0 * n_edit * 3 * total
    nnz = sum(c.nnz for c in comps)
    relight_bytes = out_bytes + 6.0 * nnz
    peak = float(peaks.get("hbm_gbs", 6800.0))
    info = plan.info()
    res = {"workload": f"{n_mesh} uneven displaced icospheres ({int(n_per.min())}-{int(n_per.max())} vertices, "
                       f"{total} in all), K={K}, J={J}, BF16 transfer, top-10 % Haar, {n_edit} edits per mesh",
           "pairs": pairs, "generator": info["generator"], "generator_param": info["param"],
           "transfer_ms": round(ms[0], 3), "transfer_g_pair_kj_per_s": round(pairs * K * J / (ms[0] * 1e-3) / 1e9, 1),
           "compress_ms": round(ms[1], 3), "relight_ms": round(ms[2], 3),
           "relight_hbm_roofline": {"bound": "hbm", "achieved": round(relight_bytes / (ms[2] * 1e-3) / 1e9, 1),
                                    "peak": peak, "unit": "GB/s",
                                    "frac": round(relight_bytes / (ms[2] * 1e-3) / 1e9 / peak, 4),
                                    "bytes": int(relight_bytes)},
           "graph_ms": round(graph_ms, 3),
           "error_vs_oracle": {"note": "M: 32 sampled rows of the 3 largest and 3 smallest meshes; B: 4 edits of the "
                                       "largest and the smallest mesh against the oracle's relight of the same "
                                       "kept coefficients"}}
    ev = res["error_vs_oracle"]
    got_m = np.concatenate([c[3] for c in m_cases], axis=2)
    f = basis.table().cpu().numpy()
    checks.add(ev, "transfer", "M", got_m, "batch_M", lambda O: np.concatenate(
        [O.transfer_rows(f, pos_h[o0:o1], area_h[o0:o1], T_h[:, o0:o1], rows) for o0, o1, rows, _ in m_cases], axis=2))
    checks.add(ev, "relight_rel", "rel_list", [c[2] for c in b_cases], "batch_B",
               lambda O: [O.relight(Cw, nu_b, g_h, light_h) for nu_b, Cw, _ in b_cases])
    del B, M, comps, g_all
    torch.cuda.empty_cache()
    return res


def energy_keep_curve(tsr, M, nu, g32, light) -> list:
    """The energy keep rule on the benchmark transfer: per retained-energy fraction, the kept share
    of the chart coefficients, the compression time (one host synchronisation inside) and the
    relative error of the relit B against keeping every coefficient (Section 5's trade-off)."""
    import torch
    full = tsr.relight(tsr.haar_compress(M, nu, 1.0), g32, light)
    K, J, _ = M.shape
    P = 1 << (nu - 1).bit_length()
    n_coef = 10 * P * P
    out = []
    for e in (0.90, 0.95, 0.98, 0.99, 0.999):
        torch.cuda.synchronize()
        t = time.perf_counter()
        comp = tsr.haar_compress_energy(M, nu, e)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t) * 1e3
        B = tsr.relight(comp, g32, light)
        err = float(((B - full).norm() / full.norm()).item())
        out.append({"energy": e, "kept_fraction": round((comp.nnz - 2 * K * J) / (K * J * n_coef), 5),
                    "compress_ms": round(ms, 3), "relight_rel_error": round(err, 6)})
    return out


def wavelet_comparison(tsr, M, nu, g32, light) -> list:
    """Relight error against keeping every coefficient, Haar vs the paper's CDF 9/7, at equal
    numbers of kept coefficients (top fraction per (k, j))."""
    full = tsr.relight(tsr.compress(M, nu, "haar", "top", 1.0), g32, light)
    out = []
    for p in (0.01, 0.05, 0.10):
        row = {"kept": p}
        for wname in ("haar", "cdf97"):
            B = tsr.relight(tsr.compress(M, nu, wname, "top", p), g32, light)
            row[wname + "_rel_error"] = round(float(((B - full).norm() / full.norm()).item()), 6)
        out.append(row)
    return out


def visibility_timing(tsr, dev) -> dict:
    """Self-shadowed SH transfer (BVH build + S = 256 rays per vertex) on the benchmark mesh."""
    import torch
    from paper_2203_12339_gb300 import scene
    w = scene.WORKLOADS[SIDE_WORKLOAD]
    mesh = scene.icosphere(w["nu"], w["amp"], w["octaves"], w["seed"])
    pos = torch.tensor(mesh.pos.astype(np.float32).T.copy(), device=dev)
    nrm = torch.tensor(mesh.normal.astype(np.float32).T.copy(), device=dev)
    tris = torch.tensor(mesh.tris.astype(np.int32), device=dev)
    S = 256
    tsr.visibility_transfer(pos, nrm, tris, w["J"], S)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    T = tsr.visibility_transfer(pos, nrm, tris, w["J"], S)
    b.record()
    torch.cuda.synchronize()
    tsr.stream_status()
    ms = a.elapsed_time(b)
    shadowed = float((T[0] < 0.97 * torch.tensor(scene.sh_transfer(mesh.normal, w["J"])[0], device=dev)).float().mean())
    return {"workload": f"{mesh.pos.shape[0]} vertices, {mesh.tris.shape[0]} triangles, J={w['J']}, S={S}",
            "ms": round(ms, 3), "g_rays_per_s": round(mesh.pos.shape[0] * S / (ms * 1e-3) / 1e9, 3),
            "shadowed_vertex_share": round(shadowed, 4)}


def reduce_max(values, world, device=None):
    """Max over ranks of a few timings (the only collective of the benchmark)."""
    if world <= 1:
        return list(values)
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def weak_scaling_value(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput in G units/s: every rank processed units_per_rank in ms (the max over ranks)."""
    return world * units_per_rank / (ms * 1e-3) / 1e9


def side_workload(tsr, dev, peaks, checks, args) -> dict:
    """The 40,962-vertex workload (K=12, J=16, amplitude 0.1): the transfer in each precision with its
    error on 1,024 sampled rows (seed 7), the energy keep rule, Haar vs CDF 9/7 and the visibility
    transfer on it."""
    import torch
    from paper_2203_12339_gb300 import scene
    w, sc = _scene(SIDE_WORKLOAD)
    K, J, N, nu = w["K"], w["J"], sc.n, w["nu"]
    sa_pca, ss_pca = scene.pca_materials(256, seed=0)
    basis, _ = tsr.fit_pca_basis(torch.tensor(sa_pca, device=dev), torch.tensor(ss_pca, device=dev), 1.3, 1024,
                                 40.0, K)
    pos_h = sc.mesh.pos.astype(np.float32)
    area_h = sc.mesh.area.astype(np.float32)
    T_h = sc.T.astype(np.float32)
    d = {"pos": torch.tensor(pos_h.T.copy(), device=dev), "area": torch.tensor(area_h, device=dev),
         "T": torch.tensor(T_h, device=dev)}
    rows = scene.sample_rows(N, 1024, seed=7)
    f = basis.table().cpu().numpy()
    precs = ("bf16",) if args.no_precision_sweep else ("bf16", "bf16x3", "fp32")
    out = {"workload": f"{SIDE_WORKLOAD}: N={N}, K={K}, J={J}",
           "transfer": transfer_sweep(tsr, basis, d, N, K, J, rows, peaks, checks, "side_rows",
                                      lambda O: O.transfer_rows(f, pos_h, area_h, T_h, rows), precs)}
    M = tsr.precompute_transfer(basis, d["pos"], d["area"], d["T"], "bf16")
    esa, ess, eeta = scene.edit_materials(64, seed=5)
    _, g32, _ = tsr.project_material(basis, torch.tensor(esa, device=dev), torch.tensor(ess, device=dev),
                                     torch.tensor(eeta, device=dev))
    light = torch.tensor(sc.light.astype(np.float32), device=dev)
    out["energy_keep_curve"] = energy_keep_curve(tsr, M, nu, g32, light)
    out["wavelet_comparison"] = wavelet_comparison(tsr, M, nu, g32, light)
    out["visibility_transfer"] = visibility_timing(tsr, dev)
    del M
    torch.cuda.empty_cache()
    return out


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2203_12339_gb300 import scene, tsr

    rank, world, local = _dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    w, sc = _scene(WORKLOAD, rank)
    N, K, J, nu = sc.n, w["K"], w["J"], w["nu"]
    sa_pca, ss_pca = scene.pca_materials(256, seed=0)
    esa, ess, eeta = scene.edit_materials(N_EDITS, seed=8)
    peaks, peak_kind = _peaks()
    checks = OracleChecks()

    # host inputs (pinned) for the end-to-end measurement
    h_pos = torch.tensor(sc.mesh.pos.astype(np.float32).T.copy()).pin_memory()
    h_area = torch.tensor(sc.mesh.area.astype(np.float32)).pin_memory()
    h_T = torch.tensor(sc.T.astype(np.float32)).pin_memory()
    h_sa = torch.tensor(esa).pin_memory()
    h_ss = torch.tensor(ess).pin_memory()
    h_eta = torch.tensor(eeta).pin_memory()
    h_light = torch.tensor(sc.light.astype(np.float32)).pin_memory()
    h_B = torch.empty((N_EDITS, 3, N), dtype=torch.float32).pin_memory()
    h_grads = torch.empty(N_EDITS * 7 + J, dtype=torch.float32).pin_memory()

    d = {k: v.to(dev) for k, v in dict(pos=h_pos, area=h_area, T=h_T, sa=h_sa, ss=h_ss, eta=h_eta,
                                         light=h_light).items()}
    M = torch.empty((K, J, N), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > L2 (129 MB)

    t0 = time.perf_counter()
    basis, _ = tsr.fit_pca_basis(torch.tensor(sa_pca, device=dev), torch.tensor(ss_pca, device=dev), 1.3, 1024,
                                 40.0, K)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3

    comp_box = [tsr.haar_compress(M, nu, KEEP)]   # handle reused by every step (tsr_haar_recompress)

    def step(inp, on_B=None):
        """The per-scene path; returns (B, gradient tensors, compressed transfer, g32).  on_B(B) runs as soon
        as B is issued."""
        _, g32, _ = tsr.project_material(basis, inp["sa"], inp["ss"], inp["eta"])
        tsr.precompute_transfer(basis, inp["pos"], inp["area"], inp["T"], "bf16", out=M)
        comp = tsr.haar_compress(M, nu, KEEP, out=comp_box[0])
        B = tsr.relight(comp, g32, inp["light"])
        if on_B is not None:
            on_B(B)
        dg, dl = tsr.relight_backward(comp, g32, inp["light"], B)          # dL/dB = B for L = 0.5 ||B||^2
        dsa, dss, de = tsr.project_material_backward(basis, inp["sa"], inp["ss"], inp["eta"], dg)
        return B, (dsa, dss, de, dl, dg), comp, g32

    d2h_stream = torch.cuda.Stream()

    def copy_B_out(B):
        # B leaves on a side stream while the adjoint runs on the main stream
        ready = torch.cuda.Event()
        ready.record()
        d2h_stream.wait_event(ready)
        with torch.cuda.stream(d2h_stream):
            h_B.copy_(B, non_blocking=True)
        B.record_stream(d2h_stream)

    def step_e2e():
        inp = {k: v.to(dev, non_blocking=True) for k, v in dict(pos=h_pos, area=h_area, T=h_T, sa=h_sa, ss=h_ss,
                                                                 eta=h_eta, light=h_light).items()}
        B, grads, _, _ = step(inp, on_B=copy_B_out)
        flat = torch.cat([g.reshape(-1).float() for g in grads[:4]])
        h_grads.copy_(flat, non_blocking=True)
        torch.cuda.current_stream().wait_stream(d2h_stream)   # B's copy joins the step

    for _ in range(args.warmup):
        step(d)
    torch.cuda.synchronize()
    tsr.stream_status()
    if world > 1:
        dist.barrier()

    stream = torch.cuda.current_stream()
    clocks = Clocks(local)
    clocks.start()
    step_ev = []
    torch.cuda.synchronize()
    tsr.kernel_timing_read()
    tsr.kernel_timing(True)          # device time of every transfer_tc_kernel launch in the timed region
    launches0 = tsr.kernel_launches()
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(d)
        b.record(stream)
        step_ev.append((a, b))
    torch.cuda.synchronize()
    launches = tsr.kernel_launches() - launches0
    tsr.kernel_timing(False)
    kernel_ms_total, kernel_n = tsr.kernel_timing_read()
    clk = clocks.stop()
    tsr.stream_status()
    ms_steps = [a.elapsed_time(b) for a, b in step_ev]
    ms_per_step = sum(ms_steps) / len(ms_steps)
    kernel_ms = kernel_ms_total / max(1, kernel_n)

    # the step's own results, compared by the oracle leg (outside the timed region)
    B, grads, comp, g32 = step(d)
    torch.cuda.synchronize()
    step_check = {"note": "one step's relit frame B (13 edits x 3 channels) and gradients dL/dg, dL/dl, "
                          "dL/dsigma_a, dL/dsigma_s, dL/deta against the oracle's relight, relight VJP and "
                          "projection VJP on the same kept coefficients and materials"}
    Cw = _dense_kept(comp, K, J).astype(np.float32)
    g_h = g32.cpu().numpy().astype(np.float64)
    light_h = sc.light.astype(np.float32)
    B_h = B.cpu().numpy()
    dsa, dss, de, dl, dg = (t.cpu().numpy() for t in grads)
    f_h = basis.table().cpu().numpy()
    checks.add(step_check, "relight_rel", "rel", B_h, "step_B", lambda O: O.relight(Cw, nu, g_h, light_h))

    def _vjp(O):
        return O.relight_vjp(Cw, nu, g_h, light_h, B_h.astype(np.float64))
    checks.add(step_check, "grad_g_rel", "rel", dg.reshape(1, -1), "step_vjp_g",
               lambda O: _vjp(O)[0].reshape(1, -1))
    checks.add(step_check, "grad_l_rel", "rel", dl.reshape(1, -1), "step_vjp_l",
               lambda O: _vjp(O)[1].reshape(1, -1))
    got_proj = np.concatenate([dsa.reshape(-1), dss.reshape(-1), de.reshape(-1)])[None, :]
    checks.add(step_check, "grad_material_rel", "rel", got_proj, "step_proj",
               lambda O: np.concatenate([x.reshape(-1) for x in O.project_material_vjp(
                   f_h, esa, ess, eeta, dg.astype(np.float64))])[None, :])
    del B, grads

    # end to end through host buffers, wall clock per step: H2D of the inputs from pinned memory, every
    # library call, D2H of B and the gradients.  Eagerly from Python (e2e.eager), and as a CUDA graph of
    # the same calls captured once and replayed per step (e2e: a render or fitting loop's launch path).
    e2e_ms = []
    for _ in range(max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        step_e2e()
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t) * 1e3)
    e2e_eager = sum(e2e_ms) / len(e2e_ms)
    e2e_mode = "CUDA graph of the whole step (H2D, library calls, D2H), replayed per step"
    try:
        g_e2e = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        cap.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cap):
            with torch.cuda.graph(g_e2e, stream=cap, capture_error_mode="thread_local"):
                step_e2e()
        torch.cuda.current_stream().wait_stream(cap)
        g_e2e.replay()
        torch.cuda.synchronize()
        tsr.stream_status()
        e2e_ms = []
        for _ in range(max(1, args.steps)):
            flush.zero_()
            torch.cuda.synchronize()
            t = time.perf_counter()
            g_e2e.replay()
            torch.cuda.synchronize()
            e2e_ms.append((time.perf_counter() - t) * 1e3)
        e2e_step = sum(e2e_ms) / len(e2e_ms)
        del g_e2e
    except RuntimeError as exc:   # capture refused: report the eager loop
        e2e_step, e2e_mode = e2e_eager, f"eager (graph capture failed: {exc})"[:200]
    h2d = sum(t.numel() * t.element_size() for t in (h_pos, h_area, h_T, h_sa, h_ss, h_eta, h_light))
    d2h = h_B.numel() * h_B.element_size() + h_grads.numel() * h_grads.element_size()

    # measurements beside the step (each with its error against the oracle, registered in `checks`)
    extra = {}
    pos_h, area_h, T_h = sc.mesh.pos.astype(np.float32), sc.mesh.area.astype(np.float32), sc.T.astype(np.float32)
    rows = scene.sample_rows(N, 64, seed=7)
    precs = ("bf16",) if args.no_precision_sweep else ("bf16", "bf16x3", "fp32")
    extra["transfer_by_precision"] = {
        "workload": f"{WORKLOAD}: N={N}, K={K}, J={J}; error on 64 sampled rows (seed 7)",
        **transfer_sweep(tsr, basis, d, N, K, J, rows, peaks, checks, "head_rows",
                         lambda O: O.transfer_rows(f_h, pos_h, area_h, T_h, rows), precs)}
    if not args.no_frame_1080p:
        tsr.precompute_transfer(basis, d["pos"], d["area"], d["T"], "bf16", out=M)
        extra["relight_frame_1080p"] = relight_frame_1080p(tsr, dev, peaks, basis, M, w, sc, checks)
    del M, flush, comp_box
    torch.cuda.empty_cache()
    if not args.no_side:
        extra["side_workload"] = side_workload(tsr, dev, peaks, checks, args)
    if not args.no_batched and world == 1:   # a one-GPU measurement of the uneven batch
        extra["batched_scene"] = batched_scene(tsr, dev, peaks, checks)

    ms_per_step, e2e_step, kernel_ms, e2e_eager_max = reduce_max([ms_per_step, e2e_step, kernel_ms, e2e_eager],
                                                                 world, dev)
    units = float(N) * N * K * J
    value = weak_scaling_value(units, world, ms_per_step)
    e2e_value = weak_scaling_value(units, world, e2e_step)
    achieved_tflops = 2.0 * units / (kernel_ms * 1e-3) / 1e12
    peak_tf = float(peaks.get("bf16_tflops_sustained", 1700.0))
    peak_burst = float(peaks.get("bf16_tflops", 1900.0))
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic (seeded displaced icosphere, SH transfer, random materials)",
        "config": {"workload": f"{WORKLOAD}: N={N}, K={K}, J={J}, {N_EDITS} RGB edits (one 1920x1080-equivalent "
                               f"frame), top-5% Haar, BF16 tensor cores with the near field in FP32",
                   "l2": "flushed between timed steps (256 MB write)",
                   "per_step": "project -> transfer(bf16) -> haar+select -> relight -> adjoint"},
        "e2e": {"value": round(e2e_value, 1), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": round(e2e_step, 3), "mode": e2e_mode,
                "eager": {"value": round(weak_scaling_value(units, world, e2e_eager_max), 1),
                          "ms_per_step": round(e2e_eager_max, 3)}},
        "gpu_launches": launches,
        "roofline": {"bound": "tensor", "achieved": round(achieved_tflops, 2), "peak": peak_tf,
                     "unit": "TFLOP/s", "frac": round(achieved_tflops / peak_tf, 4),
                     "frac_of_burst": round(achieved_tflops / peak_burst, 4),
                     "traffic": _traffic_record("transfer_tc_disp163842_traffic.json"),
                     "kernel": "transfer_tc_kernel (BF16 tcgen05 far field), per launch, CUDA events on its stream "
                               f"over the timed steps ({kernel_n} launches, {kernel_ms:.3f} ms each)",
                     "flops_per_launch": 2.0 * units,
                     "peak_kind": f"bf16 sustained ({peak_kind}; the timed region is seconds long)"},
        "transfer_kernel_ms": round(kernel_ms, 3),
        "setup_ms": round(setup_ms, 1),
        "clocks": clk,
        "step_error_vs_oracle": step_check,
    }
    line.update(extra)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(rows=args.cpu_rows)
    if rank == 0 and not args.no_oracle_errors:
        line["oracle_leg_s"] = round(checks.run(), 1)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def _cpu_threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


class _OracleCase:
    """The benchmark workload prepared once for the FP64 CPU oracle (scene, fitted basis)."""

    def __init__(self):
        from oracle import tsr_oracle as O
        from paper_2203_12339_gb300 import scene
        self.O, self.scene = O, scene
        self.w, sc = _scene(WORKLOAD)
        sa, ss = scene.pca_materials(256, seed=0)
        self.f, _ = O.fit_pca_basis(sa, ss, 1.3, 1024, 40.0, self.w["K"])
        self.n = sc.n
        self.pos = sc.mesh.pos.astype(np.float32)
        self.area = sc.mesh.area.astype(np.float32)
        self.T = sc.T.astype(np.float32)

    def run(self, rows: int, seed: int) -> tuple[float, float]:
        """Oracle transfer on `rows` sampled output vertices (all i, all k, j): (G pair.K.J/s, seconds)."""
        sel = self.scene.sample_rows(self.n, rows, seed=seed)
        t = time.perf_counter()
        self.O.transfer_rows(self.f, self.pos, self.area, self.T, sel)
        dt = time.perf_counter() - t
        return rows * self.n * self.w["K"] * self.w["J"] / dt / 1e9, dt


def cpu_baseline(rows: int = 384, seed: int = 7) -> dict:
    """FP64 oracle transfer on `rows` sampled output vertices of the same workload (all i, all k, j)."""
    case = _OracleCase()
    val, dt = case.run(rows, seed)
    w = case.w
    return {"value": round(val, 3), "unit": UNIT, "cores": _cpu_threads(), "kind": "oracle",
            "sample": f"{rows} sampled output rows x all {case.n} inputs, K={w['K']}, J={w['J']} (FP64 numpy); "
                      f"{dt:.1f} s"}


def run_reference(args):
    rank, world, _ = _dist_env()
    if rank != 0:
        return
    case = _OracleCase()
    vals, ms = [], []
    for s in range(args.warmup):
        case.run(2, seed=50 + s)
    for s in range(args.steps):
        v, dt = case.run(args.ref_rows, seed=100 + s)
        ms.append(dt * 1e3)
        vals.append(v)
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(statistics.mean(ms), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"{WORKLOAD} (oracle on sampled output rows)"},
            "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": _cpu_threads(), "kind": "oracle",
                             "sample": f"{args.ref_rows} sampled output rows x all {case.n} inputs per step"},
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-rows", type=int, default=384, help="oracle sample of the cpu_baseline leg (~10 s)")
    ap.add_argument("--ref-rows", type=int, default=16, help="oracle sample per step of --impl reference")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-errors", action="store_true", help="skip the errors against the oracle")
    ap.add_argument("--no-precision-sweep", action="store_true")
    ap.add_argument("--no-frame-1080p", action="store_true", help="skip the 13 x 163,842-vertex relight frame")
    ap.add_argument("--no-side", action="store_true", help="skip the 40,962-vertex workload")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-mesh batch (transfer, Step 2, relight)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
