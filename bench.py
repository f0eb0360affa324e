#!/usr/bin/env python
"""Local energies per second of the VQ-NQS path on GB300.

Workload (one step): E_loc of 2048 uniform random S_z = 0 samples of the
16 x 16 periodic Heisenberg model (J = 1, 512 bonds, ~258 configurations per
sample) with an 8-layer VQ transformer (d_model 256, 8 heads, codebook 256,
seeded N(0, 0.02) weights), VQ reuse on.  Every step runs the whole path:
bond enumeration, embedding, per layer LN/QKV/attention/argmin/dedupe/MLP,
head, log-ratios and the local-energy reduction.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank evaluates its own 2048
samples (weak scaling, no data-path collective); the timed region is closed by
a barrier and the max over ranks is taken.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("local energies/sec at 16×16, VQ-reuse BF16 vs plain FP32 on GB300; E_loc err vs FP64")
UNIT = "local energies/s"
WORKLOAD = dict(L=16, periodic=True, J=1.0, layers=8, d_model=256, heads=8, K=256, samples_per_gpu=2048)
FP32_FFMA_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x 2 FLOP x max SM clock
L2_FLUSH_BYTES = 256 << 20


def shard(B: int, rank: int, world: int):
    """Sample indices of one rank under weak scaling: every rank gets its own B samples."""
    return np.arange(rank * B, (rank + 1) * B)


def reduce_max(x: float, dist=None) -> float:
    if dist is None or not dist.is_initialized():
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() and
                     dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks() -> dict:
    """The measured peaks of this GPU pool, else the documented fallback."""
    try:
        m = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return {"bf16_tflops": float(m["bf16_tflops_sustained"]), "bf16_tflops_burst": float(m["bf16_tflops"]),
                "hbm_gbs": float(m["hbm_gbs"]), "src": "measured"}
    except (OSError, ValueError, KeyError):
        return {"bf16_tflops": 1700.0, "bf16_tflops_burst": 1900.0, "hbm_gbs": 6800.0, "src": "fallback"}


def stage_flops(stage: str, st: dict, w: dict, bf16: bool, inc: bool = False) -> tuple[float, str]:
    """Algorithmic FLOPs (2 per multiply-add) of one stage over the counted work, and its bound.

    Attention: 4 d FLOPs per causal query-key pair (q.k and p v over all heads);
    argmin: 2 K d per searched row; GEMMs: 6 d^2 (QKV) and 8 d^2 (each MLP GEMM)
    per unique row.  Pairs and rows are counted by the library (rows before a
    configuration's first exchanged site are not computed).  Incremental path:
    the attention stage covers the samples' own rows only; the certificate is a
    2 K d distance pass per sample row (on the BF16 path the tensor-core search's
    distances, rated like the argmin); a patch costs 8 d per (row, changed
    key) pair (two scores and two value updates per head); a recomputed row 4 d
    per query-key pair, the configurations recomputed whole likewise (their rows
    from the first changed position).  On the BF16 path the patch and the recompute run these
    products on the tensor cores and are rated against the BF16 tensor peak
    (algorithmic FLOPs: split operands take three MMAs per product, which are
    not counted); their DRAM bytes are reported beside the rate."""
    d, K, Ly = w["d_model"], w["K"], w["layers"]
    U = st["unique_rows"]
    tc = "tensor" if bf16 else "alu"
    if stage == "vq_argmin":
        rows = st["inc_searched_rows"] if inc else st["active_rows"] * Ly
        return rows * 2.0 * K * d, tc
    if stage == "attention":
        if inc:
            N = w["L"] ** 2
            return st["samples"] * Ly * N * (N + 1) / 2 * 4.0 * d, tc
        return st["attn_pairs"] * Ly * 4.0 * d, tc
    if stage == "inc_certificate":
        return st["inc_base_rows"] * 2.0 * K * d, tc
    if stage == "inc_patch":  # its scores and value sums run on the tensor cores on the BF16 path
        return st["inc_patch_pairs"] * 8.0 * d, tc
    if stage == "inc_recompute":
        return st["inc_full_pairs"] * 4.0 * d, tc
    if stage == "inc_recompute_whole":
        return st["inc_whole_pairs"] * 4.0 * d, tc
    if stage == "qkv_gemm":
        return sum(U[:Ly]) * 6.0 * d * d, tc
    if stage in ("mlp_up", "mlp_down"):
        return sum(U[1:Ly + 1]) * 8.0 * d * d, tc
    return 0.0, "hbm"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_from_profile(kernel_stage: str):
    """DRAM bytes per launch recorded by the committed ncu summary of this stage's
    kernel (profiles/traffic_<stage>.md, `key: value` lines), or None when the
    kernel source changed since it was captured."""
    path = os.path.join(ROOT, "profiles", f"traffic_{kernel_stage}.md")
    rec = {}
    try:
        for line in open(path):
            k, sep, v = line.partition(":")
            if sep and k.strip() in ("source", "source_sha256_16", "dram_bytes_per_launch"):
                rec[k.strip()] = v.strip()
    except OSError:
        return None
    src = os.path.join(ROOT, rec.get("source", ""))
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if digest != rec.get("source_sha256_16") or "dram_bytes_per_launch" not in rec:
        return None
    return float(rec["dram_bytes_per_launch"])


def cpu_oracle(spins_np, w, max_seconds=20.0, max_samples=6):
    """The FP64 oracle, as it stands, on a bounded sample of the workload."""
    import torch
    import synthetic_inputs as si
    from oracle import hamiltonian, model
    N = w["L"] ** 2
    blob = si.make_weights(N, w["layers"], w["d_model"], w["K"], seed=0)
    P = model.parse_blob(blob, N, w["layers"], w["d_model"], w["heads"], w["K"])
    t0 = time.perf_counter()
    vals = []
    for i in range(max_samples):
        vals.append(float(hamiltonian.local_energy(P, spins_np[i:i + 1], w["L"], w["periodic"], w["J"])[0]))
        if time.perf_counter() - t0 > max_seconds:
            break
    dt = time.perf_counter() - t0
    return np.array(vals), dt, torch.get_num_threads()


def run_reference(args, w):
    """The oracle timed on the host cores: each step is one sample of the workload."""
    import synthetic_inputs as si
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch
    from oracle import hamiltonian, model
    N = w["L"] ** 2
    blob = si.make_weights(N, w["layers"], w["d_model"], w["K"], seed=0)
    P = model.parse_blob(blob, N, w["layers"], w["d_model"], w["heads"], w["K"])
    spins = si.make_samples(w["L"], args.warmup + args.steps, seed=1)
    for i in range(args.warmup):
        hamiltonian.local_energy(P, spins[i:i + 1], w["L"], w["periodic"], w["J"])
    t0 = time.perf_counter()
    for i in range(args.warmup, args.warmup + args.steps):
        hamiltonian.local_energy(P, spins[i:i + 1], w["L"], w["periodic"], w["J"])
    dt = time.perf_counter() - t0
    value = args.steps / dt
    cores = torch.get_num_threads()
    sample = f"1 sample of the 16x16 workload per step (about 258 configurations, full FP64 recompute)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(w, "f64 oracle"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def config_dict(w, path):
    return {"workload": (f"{w['L']}x{w['L']} periodic Heisenberg J={w['J']:g}, {w['layers']} layers d_model "
                         f"{w['d_model']} heads {w['heads']} codebook {w['K']}, {w['samples_per_gpu']} uniform "
                         f"S_z=0 samples per GPU"),
            "path": path, "L": w["L"], "samples_per_gpu": w["samples_per_gpu"],
            "l2": "flushed between timed steps (256 MiB write); the step's working set is also far above L2"}


def gemm_probe(m, dm: int, stream=None) -> dict:
    """The QKV, MLP-up and MLP-down tensor-core GEMMs at M = 131072 (d_model dm), with single
    and with split (hi + lo, three MMA passes) operands: 3 untimed then 20 timed launches per
    shape, with the tensor fraction (of the MMAs issued) and the HBM fraction."""
    import torch
    pk = measured_peaks()
    Mg = 131072
    gemm = {"M": Mg, "peak_tflops": pk["bf16_tflops_burst"], "peak_source": f"bf16 dense, burst ({pk['src']})",
            "shapes": {}}
    for split in (False, True):
        for name, Ng, Kg, epi in (("qkv_bias_bf16", 3 * dm, dm, 0), ("mlp_up_bias_gelu_bf16", 4 * dm, dm, 1),
                                  ("mlp_down_bias_residual_f32", dm, 4 * dm, 2)):
            npl = 2 if split else 1  # operand planes (hi, lo)
            A = torch.randn(npl * Mg, Kg, device="cuda").to(torch.bfloat16)
            Bt = (0.05 * torch.randn(npl * Ng, Kg, device="cuda")).to(torch.bfloat16)
            bias = torch.zeros(Ng, device="cuda")
            Rg = torch.zeros(Mg, Ng, device="cuda") if epi == 2 else None
            Cg = torch.empty((npl if epi < 2 else 1) * Mg, Ng, dtype=torch.bfloat16 if epi < 2 else torch.float32,
                             device="cuda")
            fn = m.gemm_bf16_split if split else m.gemm_bf16
            for _ in range(3):
                fn(A, Bt, bias, epilogue=epi, R=Rg, out=Cg, stream=stream)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(20):
                fn(A, Bt, bias, epilogue=epi, R=Rg, out=Cg, stream=stream)
            a1.record(stream)
            torch.cuda.synchronize()
            sec = a0.elapsed_time(a1) / 1e3 / 20
            mma = 3 if split else 1  # BF16 MMA passes per product
            tf = 2.0 * Mg * Ng * Kg / sec / 1e12
            # bytes a launch must move: A, Bt, C (and the residual R), every plane
            nbytes = (npl * (Mg * Kg * 2 + Ng * Kg * 2) + Mg * Ng * (2 * npl if epi < 2 else 4) +
                      (Mg * Ng * 4 if epi == 2 else 0))
            gbs = nbytes / sec / 1e9
            t_tensor = mma * 2.0 * Mg * Ng * Kg / (pk["bf16_tflops_burst"] * 1e12)
            t_hbm = nbytes / (pk["hbm_gbs"] * 1e9)
            gemm["shapes"][name + ("_split" if split else "")] = {
                "N": Ng, "K": Kg, "us": sec * 1e6, "tflops": tf, "mma_tflops": mma * tf,
                "frac": mma * tf / pk["bf16_tflops_burst"], "hbm_gbs": gbs, "hbm_frac": gbs / pk["hbm_gbs"],
                "roofline_bound": "tensor" if t_tensor >= t_hbm else "hbm",
                "roofline_frac": max(t_tensor, t_hbm) / sec}
            del A, Bt, Rg, Cg
    return gemm


def vq_sweep(args) -> dict:
    """Table 1's protocol with seeded random weights: the same 16x16 network (three
    blocks and the final attention-only half-block, d_model 256, 8 attention heads,
    64 codes per quantizer head) with 1, 2 and 4 quantizer heads (6, 12, 24 bits);
    per bandwidth the unique-row fraction per layer, the FLOP reduction of the
    quantized blocks (Table 1's quantized-ops savings) and the timed local energies
    per second (FP32 reuse path; L2 flushed between steps)."""
    import torch
    import synthetic_inputs as si
    from paper_2212_11296_gb300 import REUSE, VQNQS
    L, layers, d, heads, K, B = 16, 3, 256, 8, 64, 512
    N = L * L
    blob = si.make_weights(N, layers, d, K, seed=0, half_block=True)
    spins = torch.as_tensor(si.make_samples(L, B, seed=1)).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {"workload": f"16x16 periodic Heisenberg, {layers} blocks + attention-only half-block, d_model {d} "
                       f"heads {heads}, {K} codes per quantizer head, {B} uniform S_z=0 samples",
           "flags": "reuse (FP32)",
           "data": "synthetic, seeded random weights", "bandwidths": {}}
    for H in (1, 2, 4):
        m = VQNQS(L, True, 1.0, layers, d, heads, K, blob, vq_heads=H, half_block=True)
        ws = m.workspace(REUSE)
        e = torch.empty(B, device="cuda")
        for _ in range(2):
            m.local_energy(spins, REUSE, out=e, workspace=ws)
        m.reset_stats()
        ms = []
        for _ in range(3):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            m.local_energy(spins, REUSE, out=e, workspace=ws)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        st = m.stats()
        out["bandwidths"][f"{6 * H} bits"] = {
            "vq_heads": H, "unique_row_fraction": [u / st["rows"] for u in st["unique_rows"][1:]],
            "quantized_ops_flop_reduction": st["flops_full"] / st["flops_done"], "ms_per_step": min(ms),
            "local_energies_per_s": B / (min(ms) / 1e3), "near_ties": st["near_ties"],
            "device_status": st["device_status"]}
        m.close()
    return out


def grad_bench(args) -> dict:
    """The differentiation workload: 20x20 periodic Heisenberg (N = 400, 800 bonds), 12 layers,
    d_model 384, 12 heads, codebook 512, 512 uniform S_z = 0 samples (seeded weights).  One step:
    the samples' local energies (VQ reuse, BF16 tensor-core GEMMs and attention) and the
    hand-written backward with activation recomputation giving the energy gradient
    2 mean[(E - mean E) O_k] (vqnqs_grad_log_psi).  Timed with CUDA events, L2 flushed between
    steps; reported as gradient samples per second with the two parts' times and the backward's
    per-stage times."""
    import torch
    import synthetic_inputs as si
    from paper_2212_11296_gb300 import BF16, REUSE, VQNQS
    L, layers, d, heads, K, B = 20, 12, 384, 12, 512, 512
    N = L * L
    blob = si.make_weights(N, layers, d, K, seed=0)
    spins = torch.as_tensor(si.make_samples(L, B, seed=1)).cuda()
    m = VQNQS(L, True, 1.0, layers, d, heads, K, blob)
    flags = REUSE | BF16  # (the incremental path takes d_model in {32, ..., 512} powers of two; 384 is not)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    ws = m.workspace(flags)
    for _ in range(args.warmup):
        e = m.local_energy(spins, flags, workspace=ws)
        _, g = m.grad_log_psi(spins, e_loc=e, flags=BF16)
    torch.cuda.synchronize()
    te, tg = [], []
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            e = m.local_energy(spins, flags, workspace=ws)
            ev[1].record(stream)
            _, g = m.grad_log_psi(spins, e_loc=e, flags=BF16)
            ev[2].record(stream)
            torch.cuda.synchronize()
            te.append(ev[0].elapsed_time(ev[1]))
            tg.append(ev[1].elapsed_time(ev[2]))
    m.profile(True)
    m.profile_read()
    m.local_energy(spins, flags, workspace=ws)
    prof_e = m.profile_read()
    m.grad_log_psi(spins, e_loc=e, flags=BF16)
    prof = m.profile_read()
    m.profile(False)
    _, g32 = m.grad_log_psi(spins, e_loc=e)  # the FP32 CUDA-core backward, for comparison
    torch.cuda.synchronize()
    rel32 = float((g - g32).abs().max().item() / g32.abs().max().item())
    st = m.stats()
    ms = sum(te) + sum(tg)
    stages = {k: {"ms": v[2], "launches": v[1]} for k, v in prof.items() if v[1] > 0}
    # the backward's tensor-core GEMMs, algorithmic FLOPs over the B N rows per layer: dX and dW
    # of W_qkv (2 x 6 d^2), W_o (2 x 2 d^2), W_1 and W_2 (4 x 8 d^2), and the straight-through
    # quantizer's o W^T, alpha W, alpha^T o and onehot^T dV (4 x 2 K d)
    R = B * N
    gemm_flops = layers * R * (48.0 * d * d + 8.0 * K * d)
    pk = measured_peaks()
    if "bwd_gemm" in stages and stages["bwd_gemm"]["ms"] > 0:
        tf = gemm_flops / (stages["bwd_gemm"]["ms"] / 1e3) / 1e12
        stages["bwd_gemm"].update({"flops": gemm_flops, "tflops": tf, "bound": "tensor",
                                   "frac": tf / pk["bf16_tflops"], "peak_source": f"bf16 dense, sustained ({pk['src']})"})
    return {"metric": "energy-gradient samples/sec at 20x20 (E_loc + backward)", "unit": "samples/s",
            "value": B * args.steps / (ms / 1e3), "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "eloc_ms_per_step": sum(te) / args.steps,
            "backward_ms_per_step": sum(tg) / args.steps,
            "config": {"workload": f"{L}x{L} periodic Heisenberg J=1, {layers} layers d_model {d} heads {heads} "
                                   f"codebook {K}, {B} uniform S_z=0 samples",
                       "eloc_path": "VQ-reuse BF16",
                       "backward": "hand-written, activation recomputation; GEMMs on the tensor cores with split "
                                   "BF16 operands (the dW products are one long K loop over the rows: few output "
                                   "tiles), attention backward and row-wise steps FP32 on the CUDA cores"},
            "grad_vs_fp32_backward_max_rel": rel32,
            "eloc_stages": {k: {"ms": v[2], "launches": v[1]} for k, v in prof_e.items() if v[1] > 0},
            "backward_stages": stages,
            "grad_norm": float(g.norm().item()), "device_status": st["device_status"], "clocks": clk.summary()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--flags", default="reuse,bf16,incremental,split",
                    help="comma list of reuse,bf16,incremental,split for the timed path (split: BF16 tensor-core "
                         "products from hi + lo operand pairs, FP32-grade)")
    ap.add_argument("--plain-runs", type=int, default=5, help="timed runs of the plain FP32 leg (median)")
    ap.add_argument("--chunk", type=int, default=0,
                    help="samples per chunk of the timed path's workspace (0: picked by the library's chunk-size "
                         "autotuner on the first 512 samples)")
    ap.add_argument("--samples", type=int, default=WORKLOAD["samples_per_gpu"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph replay measurement")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the incremental kernels' default work split (no vqnqs_autotune_incremental)")
    ap.add_argument("--gemm-only", action="store_true",
                    help="run only the tensor-core GEMM probe (three shapes at M = 131072) and print it")
    ap.add_argument("--grad", action="store_true",
                    help="the differentiation workload (20x20, 12 layers, d_model 384, 512 samples): E_loc plus the "
                         "energy gradient per step, printed as its own line")
    ap.add_argument("--vq-sweep", action="store_true",
                    help="quantization bandwidth sweep (Table 1 protocol, random weights): 16x16, three blocks, "
                         "64 codes per head, 1, 2 and 4 quantizer heads")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    w = dict(WORKLOAD, samples_per_gpu=args.samples)
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    import torch.distributed as dist
    import synthetic_inputs as si
    from paper_2212_11296_gb300 import BF16, BF16_SPLIT, INCREMENTAL, REUSE, VQNQS

    if args.gemm_only:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        m = VQNQS(4, True, 1.0, 1, 64, 2, 4, si.make_weights(16, 1, 64, 4))
        print(json.dumps({"gemm_tc": gemm_probe(m, w["d_model"])}))
        return 0
    if args.vq_sweep:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps(vq_sweep(args)))
        return 0
    if args.grad:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps(grad_bench(args)))
        return 0

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    flags = 0
    for f in args.flags.split(","):
        flags |= {"reuse": REUSE, "bf16": BF16, "incremental": INCREMENTAL, "split": BF16_SPLIT, "": 0}[f.strip()]
    B, L, N = w["samples_per_gpu"], w["L"], w["L"] ** 2
    blob = si.make_weights(N, w["layers"], w["d_model"], w["K"], seed=0)
    all_spins = si.make_samples(L, B * world, seed=1)
    spins_np = np.ascontiguousarray(all_spins[shard(B, rank, world)])
    m = VQNQS(L, w["periodic"], w["J"], w["layers"], w["d_model"], w["heads"], w["K"], blob)
    stream = torch.cuda.current_stream()
    spins = torch.as_tensor(spins_np).cuda()
    out = torch.empty(B, dtype=torch.float32, device="cuda")
    tuning = None
    if args.chunk <= 0:  # the library's autotuner picks the chunk size (fewer, larger launches)
        tuning = m.autotune_chunk(spins[:min(512, B)].contiguous(), flags, candidates=(8, 15, 30, 60))
        args.chunk = tuning["best"]
        m._ws.clear()
        torch.cuda.empty_cache()
    ws = m.workspace(flags, args.chunk)
    inc_tuning = None
    if (flags & INCREMENTAL) and (flags & BF16) and not args.no_tune:  # the incremental kernels' work split
        inc_tuning = m.autotune_incremental(spins[:min(512, B)].contiguous(), flags, chunk_samples=args.chunk)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        m.local_energy(spins, flags, out=out, workspace=ws)
    barrier()
    m.reset_stats()
    launches0 = m.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            m.local_energy(spins, flags, out=out, workspace=ws)
            ev[k][1].record(stream)
        barrier()
    launches = m.launch_count() - launches0
    st = m.stats()
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    t_ms = reduce_max(t_ms, dist if world > 1 else None)
    value = B * world * args.steps / (t_ms / 1e3)
    # the same steps again with the library's per-stage CUDA events on (they cost a few
    # percent, so the headline above is timed without them): stage times and the roofline
    m.profile(True)
    m.profile_read()
    barrier()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        m.local_energy(spins, flags, out=out, workspace=ws)
    barrier()
    prof = m.profile_read()
    m.profile(False)

    # end to end through the public API with host buffers
    h_spins = torch.as_tensor(spins_np).pin_memory()
    h_out = torch.empty(B, dtype=torch.float32).pin_memory()
    d_spins = torch.empty_like(spins)
    for _ in range(2):
        d_spins.copy_(h_spins, non_blocking=True)
        m.local_energy(d_spins, flags, out=out, workspace=ws)
        h_out.copy_(out, non_blocking=True)
    barrier()
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        e2e_ev[k][0].record(stream)
        d_spins.copy_(h_spins, non_blocking=True)
        m.local_energy(d_spins, flags, out=out, workspace=ws)
        h_out.copy_(out, non_blocking=True)
        e2e_ev[k][1].record(stream)
    barrier()
    e2e_ms = reduce_max(sum(a.elapsed_time(b) for a, b in e2e_ev), dist if world > 1 else None)
    e2e_value = B * world * args.steps / (e2e_ms / 1e3)
    e_gpu = h_out.numpy().astype(np.float64)

    # the same step replayed from one CUDA graph (launch overhead removed)
    graph_value = None
    if not args.no_graph:
        from paper_2212_11296_gb300 import LocalEnergyGraph
        g = LocalEnergyGraph(m, [(L, B)], flags, chunk_samples=args.chunk)
        for _ in range(2):
            g(spins)
        barrier()
        g_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            g_ev[k][0].record(stream)
            g(spins)
            g_ev[k][1].record(stream)
        barrier()
        g_ms = reduce_max(sum(a.elapsed_time(b) for a, b in g_ev), dist if world > 1 else None)
        graph_value = B * world * args.steps / (g_ms / 1e3)
        if not torch.equal(g.out, out):
            raise RuntimeError("graph replay differs from the eager step")
        del g

    # the plain full-recompute FP32 path on a subset of the same samples (median of several runs)
    n_plain = min(64, B)
    sub = spins[:n_plain].contiguous()
    ws0 = m.workspace(0)
    m.local_energy(sub, 0, workspace=ws0)
    torch.cuda.synchronize()
    plain_ms = []
    for k in range(max(1, args.plain_runs)):
        flush.fill_(k & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        m.local_energy(sub, 0, workspace=ws0)
        b.record(stream)
        torch.cuda.synchronize()
        plain_ms.append(a.elapsed_time(b))
    plain_value = n_plain / (statistics.median(plain_ms) / 1e3)

    # accuracy: the first 64 samples of the workload against the stored FP64 oracle values
    # (tests/golden/eloc_16x16_64.txt, written by a script that calls the oracle only),
    # raw: no sample exempted; the single-BF16 path beside it for context
    accuracy = None
    gold = os.path.join(ROOT, "tests", "golden", "eloc_16x16_64.txt")
    if w["L"] == 16 and B >= 64 and os.path.exists(gold):
        ref = np.loadtxt(gold, comments="#")[:, 1]
        n_acc = len(ref)
        e_acc = m.local_energy(spins[:n_acc].contiguous(), flags).cpu().numpy().astype(np.float64)
        rel = np.abs(e_acc - ref) / np.maximum(np.abs(ref), 1e-3 * N)
        bar = 2e-3 if flags & BF16 else 1e-5
        accuracy = {"max_rel": float(rel.max()), "median_rel": float(np.median(rel)), "samples": n_acc,
                    "bar": bar, "pass": bool(rel.max() <= bar),
                    "reference": "stored FP64 oracle values of the first 64 samples (no sample exempted)"}
        if flags & BF16_SPLIT:
            e1 = m.local_energy(spins[:n_acc].contiguous(), flags & ~BF16_SPLIT).cpu().numpy().astype(np.float64)
            r1 = np.abs(e1 - ref) / np.maximum(np.abs(ref), 1e-3 * N)
            accuracy["single_bf16_operands"] = {"max_rel": float(r1.max()), "median_rel": float(np.median(r1))}

    # the three per-location tensor-core GEMM shapes on a large M (the reuse
    # path only feeds them the few unique rows), each with its fused epilogue
    gemm = gemm_probe(m, w["d_model"], stream) if flags & BF16 else None

    # roofline of the dominant stage, from the live CUDA-event stage times of the
    # profiled repeat of the timed steps (same work, same stream)
    per_step = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(per_step, key=lambda k: per_step[k][2])
    calls, nl, ms = per_step[dom]
    fl, bound = stage_flops(dom, st, w, bool(flags & BF16), bool(flags & INCREMENTAL))
    pk = measured_peaks()
    if bound == "hbm":  # fl is bytes
        achieved = fl / (ms / 1e3) / 1e9 if ms > 0 else None
        peak, peak_src, unit = pk["hbm_gbs"], f"HBM copy ({pk['src']})", "GB/s"
    else:
        achieved = fl / (ms / 1e3) / 1e12 if ms > 0 else None
        unit = "TFLOP/s"
        if bound == "tensor":
            peak, peak_src = pk["bf16_tflops"], f"bf16 dense, sustained ({pk['src']})"
        else:
            peak, peak_src = FP32_FFMA_PEAK_TFLOPS, "derived: 152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz"
    roofline = {"bound": bound, "kernel": dom, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak if achieved else None, "traffic": traffic_from_profile(dom),
                "peak_source": peak_src, "launches": nl, "avg_launch_ms": ms / nl,
                "timing": "per-stage CUDA events on the launching stream over a repeat of the timed steps",
                ("bytes_per_launch" if bound == "hbm" else "flops_per_launch"): fl / max(1, nl)}
    stages = {k: {"ms_per_step": v[2] / args.steps, "launches_per_step": v[1] / args.steps,
                  "share": v[2] / max(1e-9, sum(x[2] for x in per_step.values()))} for k, v in per_step.items()}
    for k, v in per_step.items():  # each stage's algorithmic rate against its own bound
        fl_k, bound_k = stage_flops(k, st, w, bool(flags & BF16), bool(flags & INCREMENTAL))
        if fl_k > 0 and v[2] > 0:
            rate = fl_k / (v[2] / 1e3) / 1e12
            pk_k = pk["bf16_tflops"] if bound_k == "tensor" else FP32_FFMA_PEAK_TFLOPS
            stages[k].update({"tflops": rate, "bound": bound_k, "frac": rate / pk_k})

    if rank != 0:
        dist.destroy_process_group() if world > 1 else None
        return
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16" if flags & BF16 else "f32", "data": "synthetic",
        "config": config_dict(w, ("VQ-reuse" if flags & REUSE else "full recompute") +
                              (" incremental" if flags & INCREMENTAL else "") +
                              ((" BF16 tensor-core products from hi + lo operand pairs (three MMAs each, FP32 "
                                "accumulation), FP32-grade VQ" if flags & BF16_SPLIT else
                                " BF16 GEMMs, FP32 VQ") if flags & BF16 else " FP32")),
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(B * N),
                "d2h_bytes_per_step": int(B * 4)},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "graph_replay": {"value": graph_value, "unit": UNIT} if graph_value else None,
        "plain_fp32": {"value": plain_value, "unit": UNIT, "samples": n_plain, "runs": len(plain_ms),
                       "ms_runs": plain_ms},
        "err_vs_fp64": accuracy,
        "speedup_vs_plain_fp32": value / plain_value,
        "unique_row_fraction": [u / max(1, st["rows"]) for u in st["unique_rows"]],
        "flop_reduction": st["flops_full"] / max(1.0, st["flops_done"]),
        "near_ties_per_row": st["near_ties"] / max(1, st["rows"] * w["layers"]),
        "device_status": st["device_status"],
        "gemm_tc": gemm,
        "stages": stages,
        "chunk_samples": args.chunk,
        "autotune_chunk": ({"samples": min(512, B), "ms": {str(k): v for k, v in tuning["ms"].items()}}
                           if tuning else None),
        "autotune_incremental": ({"samples": min(512, B), "patch_items_per_cta": inc_tuning["patch_items"],
                                  "rows_items_per_sm": inc_tuning["rows_slices"],
                                  "patch_ms": {str(k): v for k, v in inc_tuning["patch_ms"].items()},
                                  "rows_ms": {str(k): v for k, v in inc_tuning["rows_ms"].items()}}
                                 if inc_tuning else None),
    }
    if flags & INCREMENTAL:  # row outcomes over the timed steps, summed over layers
        res["incremental"] = {k: st[k] for k in ("inc_base_rows", "inc_patched_rows", "inc_certified_rows",
                                                 "inc_full_rows", "inc_searched_rows", "inc_patch_pairs",
                                                 "inc_full_pairs", "inc_whole_pairs")}
    if world == 1 and not args.no_cpu_baseline:
        vals, dt, cores = cpu_oracle(spins_np, w)
        n = len(vals)
        rel = np.abs(e_gpu[:n] - vals) / np.maximum(np.abs(vals), 1e-3 * N)
        res["cpu_baseline"] = {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"first {n} samples of the workload, FP64 full recompute",
                               "max_rel_vs_gpu": float(rel.max())}
    print(json.dumps(res))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
