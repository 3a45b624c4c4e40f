#!/usr/bin/env python3
"""Benchmark of the 4-D spectral FNO block, forward + backward, on one GB300.

One step = fno_block_fwd_train + fno_block_bwd_saved (per-block activation
checkpointing: between the passes only the block input, the forward's
truncated spectra and GELU'(A), kept in the workspace, are held) over one batch of the
CO2-flow-like block workload: B=1, width 20, grid 128x128x128 (~2.1 M cells)
x 32 time steps, kept modes 12/12/8/8, input a seeded anisotropic smooth
Gaussian random field (correlation 20x20x4 cells, 8 steps), upstream gradient
N(0, 1).  Metric: input points x channels processed per second (Gpoint*ch/s,
B*C_in*Nx*Ny*Nz*Nt per step / step time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P] [--impl ours|reference]

The headline precision is split BF16 (bf16x3: DFT contractions on the tensor
cores as hi.hi + hi.lo + lo.hi products, FP32 accumulation).  After the timed
region the same inputs are run in FP32 (plain form), TF32 and BF16 as well; the
line carries their step times and the rel-L2 of every result against FP32.

--impl reference times the FP64 CPU oracle (the baseline arm) on a bounded
sample of the same workload (fewer channels), on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (B, C, Nx, Ny, Nz, Nt, mx, my, mz, mt, correlation lengths[, distinct channels])
    "co2_block_128c_t32": (1, 20, 128, 128, 128, 32, 12, 12, 8, 8, (20.0, 20.0, 4.0, 8.0)),
    "ns_block_64c_t16": (2, 20, 64, 64, 64, 16, 8, 8, 8, 6, (8.0, 8.0, 8.0, 8.0)),
    # the paper's own grids (CO2: 262 x 118 x 64 cells, 86 steps; Navier-Stokes:
    # 130^3 cells, 84 steps), kept modes about a fifth of each axis (mt at most
    # 8); four distinct GRF channels tiled over the width keep the host-side
    # generation short at ~170 M cells
    "co2_block_paper_262x118x64x86": (1, 20, 262, 118, 64, 86, 26, 12, 6, 8,
                                      (20.0, 20.0, 4.0, 8.0), 4),
    "ns_block_paper_130c_t84": (1, 20, 130, 130, 130, 84, 13, 13, 13, 8, (8.0, 8.0, 8.0, 8.0), 4),
}
# The Alg. 1 stacks (encoder 1x1, FNO blocks, decoder 1x1, MSE loss), one training
# pass per step:  name: (B, C_in, width, C_out, Nx, Ny, Nz, Nt, mx, my, mz, mt, blocks, inputs)
STACKS = {
    "co2_stack_128c_t32": (1, 3, 20, 1, 128, 128, 128, 32, 12, 12, 8, 8, 4, "co2"),
    "ns_stack_64c_t32": (8, 4, 32, 4, 64, 64, 64, 32, 12, 12, 12, 8, 4, "ns"),
    # small case of the CO2 stack for ncu captures (a few GB on the device)
    "co2_stack_64c_t16": (1, 3, 20, 1, 64, 64, 64, 16, 8, 8, 8, 6, 4, "co2"),
}
DEFAULT_WORKLOAD = "co2_block_128c_t32"
METRIC = "spectral block fwd+bwd Gpoint·ch/s & roofline %, BF16/split vs FP32 @ stated err"
UNIT = "Gpoint*ch/s"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            j = json.load(f)
        return {"hbm_gbs": float(j["hbm_gbs"]), "bf16_tflops": float(j["bf16_tflops"]),
                "sm_max_mhz": float(j.get("sm_max_mhz", 2070.0)), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "src": "fallback"}


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic(name, d):
    """Algorithmic (bytes, flops) of one launch of a kernel family for dims d (fwd+bwd step).

    Bytes count each tensor the kernel must read or write once; flops count the
    real multiply-adds of the separable pruned DFT GEMMs, the 1x1 linear and
    the mixing (2 flops per multiply-add).
    """
    B, Ci, Co, Nx, Ny, Nz, Nt, Jx, Jy, Jz, Jt = (d[k] for k in (
        "B", "Ci", "Co", "Nx", "Ny", "Nz", "Nt", "Jx", "Jy", "Jz", "Jt"))
    Ng = Nx * Ny * Nz * Nt
    C = Ci  # square blocks in the benchmark workloads
    grid = 4 * B * C * Ng
    t1 = 8 * B * C * Nx * Ny * Jz * Jt
    ncolz = B * C * Nx * Ny
    f_tz = ncolz * (Nz * Jt * Nt * 4 + Jz * Jt * Nz * 8)
    f_inv = B * Nx * Ny * C * (Nz * Jt * Jz * 8 + Nz * Nt * Jt * 4)
    f_lin = 2 * B * Ng * Ci * Co
    if name.startswith("fno_fwd_tz"):
        return grid + t1, f_tz
    if name.startswith("fno_epi_fwd_train"):  # training forward: writes z and GELU'(A)
        return 3 * grid + t1, f_inv + f_lin
    if name.startswith("fno_epi_fwd"):
        return 2 * grid + t1, f_inv + f_lin
    if name.startswith("fno_da_tz"):  # reads x, dz, GELU'(A); writes dA and its t,z spectrum
        return 4 * grid + t1, f_lin + f_tz
    if name.startswith("fno_da_saved"):  # reads x, dz, GELU'(A); writes dA
        return 4 * grid, f_lin
    if name.startswith("fno_epi_da"):
        return 3 * grid + t1, f_inv + 2 * f_lin
    if name.startswith("fno_epi_dx"):
        return 2 * grid + t1, f_inv + f_lin
    # the synthesis path (grids the fused epilogues do not tile, e.g. Nt = 84, 86)
    if name.startswith("fno_synth_t"):
        # inverse t to real points: reads V = [B C Nx Ny][Nz][Jt]; the forward
        # writes the output, the dX form reads and writes it (one launch of
        # each per step, so a launch averages 1.5 output tensors)
        return 8 * ncolz * Nz * Jt + 3 * grid // 2, ncolz * Nz * Nt * Jt * 4
    if name.startswith("fno_pw_add_fwd"):  # training forward: reads x and S, writes z and GELU'(A)
        return 4 * grid, f_lin
    if name.startswith("fno_pw_add_dx"):  # reads dA, writes W dA
        return 2 * grid, f_lin
    Mk = Jx * Jy * Jz * Jt
    nchunk = (B + 7) // 8  # batch chunks of the mixing kernels (W crosses HBM once per chunk)
    if name.startswith("fno_mix_adjoint"):
        return 8 * Mk * (2 * nchunk * Ci * Co + B * (2 * Ci + Co)), 16 * B * Ci * Co * Mk
    if name.startswith("fno_mix"):
        return 8 * Mk * (nchunk * Ci * Co + B * (Ci + Co)), 8 * B * Ci * Co * Mk
    return None, None


# DRAM bytes per launch per point-channel (B*C_in*N) from one ncu capture of the
# kernel at ns_block_64c_t16 (dram__bytes_read.sum + dram__bytes_write.sum),
# which scales in proportion to the units processed.  An entry is removed when
# its kernel changes.
TRAFFIC_PER_UNIT = {
    "fno_epi_fwd_train_f32": (0.804905e9 + 1.289400e9) / 167772160,
    "fno_epi_da_f32": (1.476010e9 + 0.642174e9) / 167772160,
    "fno_epi_dx_f32": (0.804837e9 + 0.609467e9) / 167772160,
    "fno_epi_da_mma_bf16x3": (1.471207e9 + 0.646687e9) / 167772160,
    "fno_epi_fwd_train_mma_bf16x3": (0.801008e9 + 1.291166e9) / 167772160,
    "fno_epi_dx_mma_bf16x3": (0.800973e9 + 0.613033e9) / 167772160,
    "fno_fwd_tz_mma_bf16x3": (0.671138e9 + 0.108852e9) / 167772160,
    "fno_epi_fwd_train_tc_bf16x3": (0.798273e9 + 1.285392e9) / 167772160,
    "fno_epi_dx_tc_bf16x3": (0.798813e9 + 0.609447e9) / 167772160,
    "fno_da_tz_bf16x3": (2.016318e9 + 0.765664e9) / 167772160,
}


def alu_peak_tflops(pk):
    """FP32 FMA peak: 152 SMs x 128 lanes x 2 flops x maximum SM clock."""
    return 152 * 128 * 2 * pk["sm_max_mhz"] * 1e6 / 1e12


def roofline_of(name, per_launch_ms, dd, pk, precision):
    """Roofline entry of one kernel: the bound (hbm, alu or tensor) with the larger fraction."""
    nbytes, nflops = algorithmic(name, dd)
    if nbytes is None:
        return None
    sec = per_launch_ms * 1e-3
    gbs = nbytes / sec / 1e9
    tfl = nflops / sec / 1e12
    f_hbm = gbs / pk["hbm_gbs"]
    if "_tc_" in name or "_mma_" in name or name.startswith(("fno_da_tz", "fno_synth_t")):
        # tensor-core kernels (mma.sync): algorithmic flops against
        # the dense BF16 peak; split BF16 issues 3 (DFT stages) or 6 (1x1
        # stages) products per real multiply-add, which the fraction leaves out
        comp = {"bound": "tensor", "achieved": round(tfl, 2), "peak": pk["bf16_tflops"],
                "unit": "TFLOP/s", "frac": round(tfl / pk["bf16_tflops"], 4),
                "peak_src": pk["src"] + " cuBLAS bf16 burst"}
    else:
        ap = alu_peak_tflops(pk)
        comp = {"bound": "alu", "achieved": round(tfl, 2), "peak": round(ap, 1), "unit": "TFLOP/s",
                "frac": round(tfl / ap, 4),
                "peak_src": "FP32 FMA: 152 SMs x 128 lanes x 2 flops x max SM clock"}
    hbm = {"bound": "hbm", "achieved": round(gbs, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
           "frac": round(f_hbm, 4), "peak_src": pk["src"] + " copy bandwidth"}
    best, other = (hbm, comp) if f_hbm >= comp["frac"] else (comp, hbm)
    out = dict(best)
    tpu = TRAFFIC_PER_UNIT.get(name)
    units = dd["B"] * dd["Ci"] * dd["Nx"] * dd["Ny"] * dd["Nz"] * dd["Nt"]
    out.update({"traffic": round(tpu * units) if tpu else None,
                "traffic_src": "ncu dram bytes at ns_block_64c_t16, scaled by units" if tpu else None,
                "kernel": name, "ms_per_launch": round(per_launch_ms, 4),
                "alg_bytes": nbytes, "alg_flops": nflops,
                "other": {k: other[k] for k in ("bound", "achieved", "peak", "unit", "frac")}})
    return out


def sample_points(grid, n, seed):
    """n grid points (x, y, z, t): the two ends of every axis through the centre,
    the first and the last corner, then seeded random points."""
    import numpy as np
    g = np.random.Generator(np.random.PCG64(seed))
    pts = np.stack([g.integers(0, s, n) for s in grid], axis=1)
    edges = []
    for a, s in enumerate(grid):
        for v in (0, s - 1):
            p = [s2 // 2 for s2 in grid]
            p[a] = v
            edges.append(p)
    edges.append([0, 0, 0, 0])
    edges.append([s - 1 for s in grid])
    return np.concatenate([np.array(edges, dtype=np.int64), pts.astype(np.int64)])[:n]


def oracle_reference(dims, x, w, wl, b, dz, pts):
    """The FP64 oracle's block forward and backward on the same inputs: z and dx at
    the sampled points, dw, dw_lin and db in full (the kept spectra are exact)."""
    import oracle
    _, zp = oracle.block_fwd(dims, x, w, wl, b, full=False, pts=pts)
    r = oracle.block_bwd(dims, x, w, dz, wl, b, full=False, pts=pts)
    return {"z": zp, "dx": r["dx_pts"], "dw": r["dw"], "dw_lin": r["dwl"], "db": r["db"]}


def errors_vs_oracle(ref, outs, pts):
    """rel-L2 per tensor of the GPU results against the oracle reference."""
    import numpy as np
    import torch
    z, dx, dw, dwl, db = outs
    ix = [torch.from_numpy(pts[:, a]).to(z.device) for a in range(4)]
    got = {"z": z[:, :, ix[0], ix[1], ix[2], ix[3]], "dx": dx[:, :, ix[0], ix[1], ix[2], ix[3]],
           "dw": dw, "dw_lin": dwl, "db": db}
    out = {}
    for k, r in ref.items():
        a = got[k].detach().double().cpu().numpy().ravel()
        out[k] = float(np.linalg.norm(a - r.ravel()) / np.linalg.norm(r.ravel()))
    return out


def precision_sweep(args, step_of, outs, stream, barrier, units, ref=None, pts=None, check=None):
    """Time every precision on the resident inputs; rel-L2 of every result against
    the FP64 oracle (ref, at the sampled points pts) and against the FP32 plain form.
    check() raises if a bounded device-side wait of the timed steps gave up."""
    import torch
    ref_prec = "fp32"
    runs = {}
    ref32 = None
    for prec in ["fp32", "tf32", "bf16", "bf16x3"]:
        st = step_of(prec)
        for _ in range(3):
            st()
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            st()
        b.record(stream)
        barrier()
        if check is not None:
            check()
        ms = a.elapsed_time(b) / args.steps
        res = [t.detach().double().clone() if prec == ref_prec else t.detach().double() for t in outs]
        if prec == ref_prec:
            ref32 = res
            err = None
        else:
            err = {k: float(torch.linalg.vector_norm(r - q) / torch.linalg.vector_norm(q))
                   for k, r, q in zip(("z", "dx", "dw", "dw_lin", "db"), res, ref32)}
        runs[prec] = {"ms_per_step": round(ms, 3), "value": units / (ms * 1e-3) / 1e9,
                      "rel_l2_vs_oracle": errors_vs_oracle(ref, outs, pts) if ref is not None else None,
                      "rel_l2_vs_fp32": err}
        del res
    runs["tolerance_vs_oracle"] = {"fp32": 1e-5, "bf16x3": 1e-5, "bf16": 2e-2, "tf32": 5e-3}
    runs["note"] = ("rel-L2 vs the FP64 oracle: z and dx at the sampled points, dw, dw_lin, db "
                    "in full; the tf32 bound is ten TF32-rounded operands on a path (2^-11 each)")
    return runs


def replica_seed(rank: int) -> int:
    """Input-configuration index of a replica: independent replicas draw different seeds."""
    return 4 + rank


def reduce_step_time(ms: float, dist=None, device=None) -> float:
    """Max of the per-rank step times (the slowest replica sets the job's pace)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank: int, world: int, ms: float) -> float:
    """Gpoint*ch/s of the whole job: every rank's units over the slowest step time."""
    return units_per_rank * world / (ms * 1e-3) / 1e9


# The CPU baseline times the whole oracle block fwd + bwd (kept spectra, mixing,
# the z synthesis, 1x1, bias, GELU, and every gradient including the dX synthesis
# with its W_lin dA term) with every channel of the workload, on a bounded cut of
# its grid: at most 64 x 32 x 32 cells in x, y, z, every time step, the same kept
# modes.  About 5-10 s per pass on 16 host cores.
CPU_SAMPLE_GRID = (64, 32, 32)


def oracle_sample_time(wl_name, seed=1000):
    """Seconds of one full oracle fwd+bwd on the bounded sample, its units and description."""
    import oracle
    from oracle import Dims
    from paper_2211_12709_gb300 import inputs
    B, C, Nx, Ny, Nz, Nt, mx, my, mz, mt, ell = WORKLOADS[wl_name][:11]
    nx, ny, nz = (min(n, c) for n, c in zip((Nx, Ny, Nz), CPU_SAMPLE_GRID))
    d = Dims(1, C, C, nx, ny, nz, Nt, mx, my, mz, mt)
    x = inputs.normal((1, C) + d.grid, seed)
    w = inputs.spectral_weights(C, C, d.modes, seed + 1)
    wl, b = inputs.linear_params(C, C, seed + 2)
    dz = inputs.normal((1, C) + d.grid, seed + 3)
    cores = oracle.threads()
    t0 = time.perf_counter()
    oracle.block_fwd(d, x, w, wl, b, full=True)
    oracle.block_bwd(d, x, w, dz, wl, b, full=True)
    dt = time.perf_counter() - t0
    units = d.B * d.Ci * d.n_grid
    sample = (f"the whole FP64 oracle block fwd+bwd (z and dX syntheses, 1x1, GELU, every gradient), "
              f"B=1, C_in=C_out={C} (every channel), grid {nx}x{ny}x{nz}x{Nt} cut from "
              f"{Nx}x{Ny}x{Nz}x{Nt}, modes {mx}/{my}/{mz}/{mt}")
    return dt, units, cores, sample


def stack_arrays(name, cfg, width=None, batch=None):
    """Seeded input, target and parameters of a stack workload (NumPy, float32)."""
    from paper_2211_12709_gb300 import inputs
    B, C0, W, Co, Nx, Ny, Nz, Nt, mx, my, mz, mt, L, kind = STACKS[name]
    B = batch or B
    W = width or W
    grid = (Nx, Ny, Nz, Nt)
    gen = inputs.co2_stack_inputs if kind == "co2" else inputs.ns_stack_inputs
    x0, target = gen(B, grid, inputs.SEED_INPUT + cfg)
    enc = inputs.linear_params(C0, W, inputs.SEED_LINEAR + cfg)
    blocks = []
    for k in range(L):
        w = inputs.spectral_weights(W, W, (2 * mx, 2 * my, 2 * mz, mt), inputs.SEED_SPECTRAL_W + cfg + k)
        wl, bb = inputs.linear_params(W, W, inputs.SEED_LINEAR + cfg + 10 + k)
        blocks.append((w, wl, bb))
    dec = inputs.linear_params(W, Co, inputs.SEED_LINEAR + cfg + 20)
    return x0, target, enc, blocks, dec


def oracle_stack_time(name, width=2, seed=0):
    """Seconds of one oracle training pass of a stack on its grid with a narrower width."""
    import oracle
    from oracle import Dims
    B, C0, W, Co, Nx, Ny, Nz, Nt, mx, my, mz, mt, L, kind = STACKS[name]
    x0, target, enc, blocks, dec = stack_arrays(name, seed, width=width, batch=1)
    d = Dims(1, width, width, Nx, Ny, Nz, Nt, mx, my, mz, mt)
    cores = oracle.threads()
    t0 = time.perf_counter()
    oracle.stack_loss_and_grads(d, x0, target, enc, blocks, dec)
    dt = time.perf_counter() - t0
    units = width * d.n_grid * L
    return dt, units, cores, (f"B=1, width {width} (C_in {C0}, C_out {Co}), {L} blocks on the "
                              f"{Nx}x{Ny}x{Nz}x{Nt} grid, modes {mx}/{my}/{mz}/{mt}")


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    if args.workload in STACKS:
        dts = []
        if args.warmup > 0:
            oracle_stack_time(args.workload)
        for _ in range(args.steps):
            dt, units, cores, sample = oracle_stack_time(args.workload)
            dts.append(dt)
        tot = sum(dts)
        value = units * len(dts) / tot / 1e9
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(dts),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }), flush=True)
        return 0
    wl_name = args.workload
    B, C, Nx, Ny, Nz, Nt, mx, my, mz, mt, ell = WORKLOADS[wl_name][:11]
    if args.warmup > 0:  # one untimed oracle pass stands for the warm-up steps
        oracle_sample_time(wl_name)
    times = []
    units = cores = sample = None
    for _ in range(args.steps):
        dt, units, cores, sample = oracle_sample_time(wl_name)
        times.append(dt)
    tot = sum(times)
    value = units * len(times) / tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl_name, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_stack(args, rank, world, local, dev, dist):
    """One training pass of an Alg. 1 stack per step, through StackRunner (C ABI only)."""
    import numpy as np
    import torch

    from paper_2211_12709_gb300 import _lib
    from paper_2211_12709_gb300.stack import StackRunner

    B, C0, W, Co, Nx, Ny, Nz, Nt, mx, my, mz, mt, L, kind = STACKS[args.workload]
    grid = (Nx, Ny, Nz, Nt)
    Ng = Nx * Ny * Nz * Nt
    cfg = replica_seed(rank)
    x0_np, tg_np, enc, blocks, dec = stack_arrays(args.workload, cfg)
    x0_h = torch.from_numpy(x0_np).pin_memory()
    tg_h = torch.from_numpy(tg_np).pin_memory()
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    params = {"enc_w": T(enc[0]), "enc_b": T(enc[1]), "dec_w": T(dec[0]), "dec_b": T(dec[1]),
              "blocks": [tuple(T(a) for a in blk) for blk in blocks]}
    x0 = x0_h.to(dev)
    tg = tg_h.to(dev)
    runner = StackRunner(B, C0, grid, params, (mx, my, mz, mt), args.precision, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    run = (lambda: runner.train_step(x0, tg, lr=1e-4)) if args.train else (lambda: runner.step(x0, tg))
    for _ in range(args.warmup):
        run()
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    n0 = _lib.fno_launch_count()
    _lib.fno_profile_start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        run()
    e1.record(stream)
    barrier()
    prof = _lib.fno_profile_stop()
    launches = _lib.fno_launch_count() - n0
    clocks = sampler.stop()
    ms = reduce_step_time(e0.elapsed_time(e1) / args.steps, dist, dev)
    units = B * W * Ng * L  # point-channels through the blocks per step
    value = whole_job_value(units, world, ms)
    loss = float(runner.loss.item())

    e2e = None
    if not args.no_e2e:
        grads = [runner.grads["enc_w"], runner.grads["enc_b"], runner.grads["dec_w"],
                 runner.grads["dec_b"]] + [t for blk in runner.grads["blocks"] for t in blk]
        outs = [runner.loss] + grads
        outs_h = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in outs]
        h2d = (x0_h.numel() + tg_h.numel()) * 4
        d2h = sum(t.numel() * 4 for t in outs_h)
        k2 = max(2, min(args.steps, 5))
        barrier()
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        for _ in range(k2):
            x0.copy_(x0_h, non_blocking=True)
            tg.copy_(tg_h, non_blocking=True)
            run()
            for hb, db_ in zip(outs_h, outs):
                hb.copy_(db_, non_blocking=True)
        e3.record(stream)
        barrier()
        ms2 = reduce_step_time(e2.elapsed_time(e3) / k2, dist, dev)
        e2e = {"value": whole_job_value(units, world, ms2), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ms2}

    pk = peaks()
    dd = {"B": B, "Ci": W, "Co": W, "Nx": Nx, "Ny": Ny, "Nz": Nz, "Nt": Nt,
          "Jx": 2 * mx, "Jy": 2 * my, "Jz": 2 * mz, "Jt": mt}
    tot_prof = sum(v[1] for v in prof.values()) if prof else 0.0
    kernel_share = {}
    for k, (n, t) in sorted(prof.items(), key=lambda kv: -kv[1][1]):
        r = roofline_of(k, t / n, dd, pk, args.precision)
        kernel_share[k] = {"launches": n, "ms": round(t, 4),
                           "share": round(t / tot_prof, 4) if tot_prof else None,
                           "bound": r["bound"] if r else None, "frac": r["frac"] if r else None}
    top = max(prof.items(), key=lambda kv: kv[1][1]) if prof else None
    roof = roofline_of(top[0], top[1][1] / top[1][0], dd, pk, args.precision) if top else None

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            dt, u, cores, sample = oracle_stack_time(args.workload)
            cpu = {"value": u / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
        except Exception as ex:  # the baseline is reported, never required
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": f"failed: {ex}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "tf32": "tf32+f32", "bf16": "bf16+f32",
                                           "bf16x3": "bf16x3+f32"}[args.precision],
            "data": "synthetic",
            "config": {"workload": args.workload, "B": B, "C_in": C0, "width": W, "C_out": Co,
                       "blocks": L, "grid": list(grid), "modes": [mx, my, mz, mt],
                       "precision": args.precision,
                       "step": ("encoder 1x1+GELU, FNO blocks, decoder 1x1+GELU, MSE loss; forward "
                                "and backward (Alg. 1); block inputs and truncated spectra kept"
                                + ("; Adam update of every parameter" if args.train else "")),
                       "units": "B*width*N per block, summed over the blocks",
                       "l2": "activations larger than L2; no flush",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "loss": loss, "bytes_held": runner.bytes_held(),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "kernels": kernel_share,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


SMALL_WORKLOAD = "ns_block_64c_t16"


def workload_arrays(name, cfg):
    """Seeded input, upstream gradient and parameters of a block workload (NumPy, FP32)."""
    import numpy as np
    from paper_2211_12709_gb300 import inputs
    B, C, Nx, Ny, Nz, Nt, mx, my, mz, mt, ell = WORKLOADS[name][:11]
    n_distinct = WORKLOADS[name][11] if len(WORKLOADS[name]) > 11 else C
    x = inputs.grf((B, n_distinct), (Nx, Ny, Nz, Nt), ell, inputs.SEED_INPUT + cfg)
    if n_distinct < C:
        x = np.tile(x, (1, (C + n_distinct - 1) // n_distinct, 1, 1, 1, 1))[:, :C].copy()
    dz = inputs.normal((B, C, Nx, Ny, Nz, Nt), inputs.SEED_UPSTREAM + cfg)
    w = inputs.spectral_weights(C, C, (2 * mx, 2 * my, 2 * mz, mt), inputs.SEED_SPECTRAL_W + cfg)
    wl, b = inputs.linear_params(C, C, inputs.SEED_LINEAR + cfg)
    return x, dz, w, wl, b


def shape_sweep(name, args, dev, stream, barrier, cfg):
    """The precision sweep (training forward + saved backward, every precision,
    times and errors against the FP64 oracle) on another block workload."""
    import torch
    from oracle import Dims
    from paper_2211_12709_gb300 import _lib, ops
    B, C, Nx, Ny, Nz, Nt, mx, my, mz, mt, ell = WORKLOADS[name][:11]
    x_np, dz_np, w_np, wl_np, b_np = workload_arrays(name, cfg)
    T = lambda a: torch.from_numpy(a).to(dev)
    x, dz, w, wl, bias = T(x_np), T(dz_np), T(w_np), T(wl_np), T(b_np)
    z, dx, dw, dwl, db = (torch.empty_like(t) for t in (x, x, w, wl, bias))
    d = ops.dims_of(x, C, (mx, my, mz, mt))
    nws = max(_lib.fno_workspace_bytes(d, ops.precision_code(q), ops.OP_BLOCK_TRAIN)
              for q in ("fp32", "tf32", "bf16", "bf16x3"))
    ws = torch.empty(nws, dtype=torch.uint8, device=dev)
    sh = int(stream.cuda_stream)

    def step_of(prec, saved=True):
        pc = ops.precision_code(prec)

        def st():
            _lib.fno_block_fwd_train(d, pc, x.data_ptr(), w.data_ptr(), wl.data_ptr(), bias.data_ptr(),
                                     z.data_ptr(), ws.data_ptr(), nws, sh)
            _lib.fno_block_bwd_saved(d, pc, x.data_ptr(), w.data_ptr(), wl.data_ptr(), bias.data_ptr(),
                                     dz.data_ptr(), dx.data_ptr(), dw.data_ptr(), dwl.data_ptr(),
                                     db.data_ptr(), ws.data_ptr(), nws, sh)
        return st

    pts = sample_points((Nx, Ny, Nz, Nt), 96, 78)
    ref = oracle_reference(Dims(B, C, C, Nx, Ny, Nz, Nt, mx, my, mz, mt), x_np, w_np, wl_np, b_np, dz_np, pts)
    out = precision_sweep(args, step_of, (z, dx, dw, dwl, db), stream, barrier, B * C * Nx * Ny * Nz * Nt,
                          ref, pts, check=lambda: _lib.fno_workspace_status(ws.data_ptr(), sh))
    out["config"] = {"B": B, "C_in": C, "C_out": C, "grid": [Nx, Ny, Nz, Nt], "modes": [mx, my, mz, mt]}
    del x, dz, z, dx, ws
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["fp32", "tf32", "bf16", "bf16x3"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + sorted(STACKS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--train", action="store_true",
                    help="stack workloads: each step also takes an Adam update of every parameter")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    from paper_2211_12709_gb300 import _lib, inputs, ops

    assert torch.cuda.is_available(), "bench.py needs a CUDA GPU"
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    if args.workload in STACKS:
        return run_stack(args, rank, world, local, dev, dist)

    B, C, Nx, Ny, Nz, Nt, mx, my, mz, mt, ell = WORKLOADS[args.workload][:11]
    modes = (mx, my, mz, mt)
    Ng = Nx * Ny * Nz * Nt
    cfg = replica_seed(rank)
    # inputs in pinned host memory (the e2e leg copies them every step)
    x_np, dz_np, w_np, wl_np, b_np = workload_arrays(args.workload, cfg)
    x_h = torch.from_numpy(x_np).pin_memory()
    dz_h = torch.from_numpy(dz_np).pin_memory()
    del x_np, dz_np
    w = torch.from_numpy(w_np).to(dev)
    wl, bias = torch.from_numpy(wl_np).to(dev), torch.from_numpy(b_np).to(dev)
    x = x_h.to(dev)
    dz = dz_h.to(dev)
    z = torch.empty_like(x)
    dx = torch.empty_like(x)
    dw = torch.empty_like(w)
    dwl = torch.empty_like(wl)
    db = torch.empty_like(bias)
    d = ops.dims_of(x, C, modes)
    p = ops.precision_code(args.precision)
    nws = max(_lib.fno_workspace_bytes(d, ops.precision_code(q), op)
              for q in ("fp32", "tf32", "bf16", "bf16x3")
              for op in (ops.OP_BLOCK_FWD, ops.OP_BLOCK_BWD, ops.OP_BLOCK_TRAIN))
    ws = torch.empty(nws, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    sh = int(stream.cuda_stream)

    def step_of(prec, saved=True):
        """Forward + backward.  saved: fno_block_fwd_train, then the backward reuses
        the forward's spectra and GELU'(A) from ws; else fno_block_fwd and the
        backward recomputes them from x."""
        pc = ops.precision_code(prec)
        fwd = _lib.fno_block_fwd_train if saved else _lib.fno_block_fwd
        bwd = _lib.fno_block_bwd_saved if saved else _lib.fno_block_bwd

        def st():
            fwd(d, pc, x.data_ptr(), w.data_ptr(), wl.data_ptr(), bias.data_ptr(),
                z.data_ptr(), ws.data_ptr(), nws, sh)
            bwd(d, pc, x.data_ptr(), w.data_ptr(), wl.data_ptr(), bias.data_ptr(), dz.data_ptr(),
                dx.data_ptr(), dw.data_ptr(), dwl.data_ptr(), db.data_ptr(), ws.data_ptr(), nws, sh)
        return st

    step = step_of(args.precision)

    def step_on(bufs):
        """The step on another buffer set (x, dz, z, dx, dw, dwl, db)."""
        pc = ops.precision_code(args.precision)
        xb, dzb, zb, dxb, dwb, dwlb, dbb = bufs

        def st():
            _lib.fno_block_fwd_train(d, pc, xb.data_ptr(), w.data_ptr(), wl.data_ptr(),
                                     bias.data_ptr(), zb.data_ptr(), ws.data_ptr(), nws, sh)
            _lib.fno_block_bwd_saved(d, pc, xb.data_ptr(), w.data_ptr(), wl.data_ptr(),
                                     bias.data_ptr(), dzb.data_ptr(), dxb.data_ptr(),
                                     dwb.data_ptr(), dwlb.data_ptr(), dbb.data_ptr(),
                                     ws.data_ptr(), nws, sh)
        return st

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    barrier()

    # ---- device-resident timed region ----
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    n0 = _lib.fno_launch_count()
    _lib.fno_profile_start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    prof = _lib.fno_profile_stop()
    # a bounded device-side wait that gave up would void the timing: raise
    _lib.fno_workspace_status(ws.data_ptr(), sh)
    launches = _lib.fno_launch_count() - n0
    clocks = sampler.stop()
    ms = reduce_step_time(e0.elapsed_time(e1) / args.steps, dist, dev)
    units = B * C * Ng
    value = whole_job_value(units, world, ms)

    # the same step with the backward recomputing the forward spectra from x
    step_rc = step_of(args.precision, saved=False)
    for _ in range(2):
        step_rc()
    barrier()
    e4 = torch.cuda.Event(enable_timing=True)
    e5 = torch.cuda.Event(enable_timing=True)
    e4.record(stream)
    for _ in range(args.steps):
        step_rc()
    e5.record(stream)
    barrier()
    ms_rc = reduce_step_time(e4.elapsed_time(e5) / args.steps, dist, dev)

    # ---- end to end: pinned host inputs -> C ABI -> host results ----
    # Every step copies its inputs from pinned host memory and its results back.
    # The copies run on their own streams with two device buffer sets, so step
    # i's uploads and step i - 1's downloads overlap the compute of the steps
    # beside them (as an input pipeline feeding the library would).
    e2e = None
    if not args.no_e2e:
        sets = [(x, dz, z, dx, dw, dwl, db)]
        sets.append(tuple(torch.empty_like(t) for t in sets[0]))
        outs_h = [[torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in st[2:]]
                  for st in sets]
        h2d = (x_h.numel() + dz_h.numel()) * 4
        d2h = sum(t.numel() * 4 for t in outs_h[0])
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        steps_on = [step_on(st) for st in sets]
        k2 = max(2, min(args.steps, 5))
        ev_in = [torch.cuda.Event() for _ in sets]
        ev_done = [torch.cuda.Event() for _ in sets]
        ev_out = [torch.cuda.Event() for _ in sets]

        def pipeline(k):
            """k steps, each uploading its inputs and downloading its results;
            returns the (start, end) events on the compute stream."""
            e_a = torch.cuda.Event(enable_timing=True)
            e_b = torch.cuda.Event(enable_timing=True)
            e_a.record(stream)
            s_in.wait_event(e_a)
            for i in range(k):
                j = i % 2
                xs, dzs = sets[j][0], sets[j][1]
                with torch.cuda.stream(s_in):
                    if i >= 2:
                        s_in.wait_event(ev_done[j])     # step i - 2 no longer reads this set
                    xs.copy_(x_h, non_blocking=True)
                    dzs.copy_(dz_h, non_blocking=True)
                    ev_in[j].record(s_in)
                stream.wait_event(ev_in[j])
                if i >= 2:
                    stream.wait_event(ev_out[j])        # step i - 2's results have left the device
                steps_on[j]()
                ev_done[j].record(stream)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_done[j])
                    for hb, dbuf in zip(outs_h[j], sets[j][2:]):
                        hb.copy_(dbuf, non_blocking=True)
                    ev_out[j].record(s_out)
            for j in range(len(sets)):
                stream.wait_event(ev_out[j])
            e_b.record(stream)
            return e_a, e_b

        # untimed warm-up of the pipeline: the first copies into fresh pinned
        # buffers and the first launches on the second buffer set are slower
        pipeline(2)
        barrier()
        e2, e3 = pipeline(k2)
        barrier()
        ms2 = reduce_step_time(e2.elapsed_time(e3) / k2, dist, dev)
        e2e = {"value": whole_job_value(units, world, ms2), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ms2,
               "pipelined": "uploads, compute and downloads on three streams, two buffer sets"}
        del sets[1], outs_h

    # ---- roofline of the dominant kernel ----
    pk = peaks()
    dd = {"B": B, "Ci": C, "Co": C, "Nx": Nx, "Ny": Ny, "Nz": Nz, "Nt": Nt,
          "Jx": 2 * mx, "Jy": 2 * my, "Jz": 2 * mz, "Jt": mt}
    kernel_share = {}
    tot_prof = sum(v[1] for v in prof.values()) if prof else 0.0
    for k, (n, t) in sorted(prof.items(), key=lambda kv: -kv[1][1]):
        r = roofline_of(k, t / n, dd, pk, args.precision)
        kernel_share[k] = {"launches": n, "ms": round(t, 4),
                           "share": round(t / tot_prof, 4) if tot_prof else None,
                           "bound": r["bound"] if r else None, "frac": r["frac"] if r else None}
    top = max(prof.items(), key=lambda kv: kv[1][1]) if prof else None
    roof = roofline_of(top[0], top[1][1] / top[1][0], dd, pk, args.precision) if top else None

    # ---- every precision on the same inputs: time, and error vs the FP64 oracle ----
    sweep = None
    if not args.no_sweep:
        from oracle import Dims
        od = Dims(B, C, C, Nx, Ny, Nz, Nt, mx, my, mz, mt)
        pts = sample_points((Nx, Ny, Nz, Nt), 96, 77)
        ref = oracle_reference(od, x_h.numpy(), w_np, wl_np, b_np, dz_h.numpy(), pts)
        sweep = precision_sweep(args, step_of, (z, dx, dw, dwl, db), stream, barrier, units * world,
                                ref, pts, check=lambda: _lib.fno_workspace_status(ws.data_ptr(), sh))
        if args.workload != SMALL_WORKLOAD:
            sweep[SMALL_WORKLOAD] = shape_sweep(SMALL_WORKLOAD, args, dev, stream, barrier, cfg)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            dt, u, cores, sample = oracle_sample_time(args.workload)
            cpu = {"value": u / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
        except Exception as ex:  # the baseline is reported, never required
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": f"failed: {ex}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "tf32": "tf32+f32", "bf16": "bf16+f32",
                                           "bf16x3": "bf16x3+f32"}[args.precision],
            "data": "synthetic",
            "config": {"workload": args.workload, "B": B, "C_in": C, "C_out": C,
                       "grid": [Nx, Ny, Nz, Nt], "modes": [mx, my, mz, mt], "precision": args.precision,
                       "step": "fno_block_fwd_train + fno_block_bwd_saved (the backward reuses "
                               "the forward's truncated spectra and GELU'(A), kept in the "
                               "workspace)",
                       "recompute_ms_per_step": round(ms_rc, 4),
                       "l2": f"inputs larger than L2 ({4 * B * C * Ng / 1e9:.1f} GB per tensor); no flush",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "kernels": kernel_share, "precision_sweep": sweep,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
