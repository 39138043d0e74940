#!/usr/bin/env python
"""Sweeps/s of the worldline FFBS + Hirsch-Gibbs sweep on synthetic Hubbard lattices.

Workload (one step = one sweep of the whole batch: anchor draw, FFBS of every
worldline, Gibbs resample of every field, observable accumulation):
  L=32 (N=1024), t=1, U=4, beta=4, dtau=0.05 (M=80), half filling (512 up + 512 down
  worldlines), 64 independent chains with Philox seeds 0..63 (offset 64*rank per rank),
  batched FP32 filter with FP64 log-normaliser, one CUDA-graph replay per sweep.

Printed beside it on the same JSON line: the FFBS kernel's roofline from CUDA events
taken live around its launches, the plain FP64 form (same kernels in double, one launch
per phase, no graph), the end-to-end rate through the public API with host buffers,
and the CPU oracle timed on a bounded sample on this host's cores.

--impl reference times the CPU oracle (the test oracle of this repository, FP64) on a
bounded sample of the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORK = dict(L=32, t=1.0, U=4.0, beta=4.0, dtau=0.05, filling=1.0, chains=64)
METRIC = "sweeps/s at L=32 (batched FP32 vs plain FP64 GPU, same accuracy); % HBM roofline"
WORKLOAD = ("2D Hubbard L=32 (N=1024) t=1 U=4 beta=4 dtau=0.05 (M=80) half filling, "
            "512+512 worldlines x 64 chains, Philox seeds 0..63; FP32 FFT filter, FP64 log Z")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured", d.get("sm_max_mhz", 2070.0)
    return 6800.0, "fallback", 2070.0


def start_clocks(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                                stdout=f, stderr=subprocess.DEVNULL), f
    except Exception:
        return None, None


def stop_clocks(proc, f, path, device):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except Exception:
        proc.kill()
    f.close()
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9 or parts[0] != str(device):
            continue
        try:
            sm.append(float(parts[1]))
            mx = float(parts[2])
        except ValueError:
            continue
        for n, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_sample(target_s=12.0):
    """Time the FP64 oracle (OpenMP over worldlines) on the first k worldlines of each
    spin of chain 0 for one sweep, k grown until the sweep takes at least half of
    target_s (after an untimed warm-up sweep); extrapolate per worldline to the whole
    64-chain batch."""
    import oracle

    w = WORK
    args = (w["L"], w["t"], w["U"], w["beta"], w["dtau"], w["filling"], 0)
    cores = oracle.num_threads()
    step = max(1, cores // 2)  # 2 step worldlines: one per thread
    oracle.Chain(*args).sweep(nwl_limit=step)  # library load, thread pool start
    k2 = step
    while True:
        orc2 = oracle.Chain(*args)
        t0 = time.perf_counter()
        orc2.sweep(nwl_limit=k2)
        dt2 = time.perf_counter() - t0
        if dt2 >= 0.5 * target_s or k2 >= orc2.Nsig:
            break
        k2 = min(orc2.Nsig, max(k2 + step, int(k2 * target_s / max(dt2, 1e-3)) // step * step))
    per_wl = dt2 / (2 * k2)
    total_wl = w["chains"] * 2 * orc2.Nsig
    return {"value": 1.0 / (per_wl * total_wl), "unit": "sweeps/s", "cores": cores, "kind": "oracle",
            "rate_kind": "per-worldline rate extrapolated from a sample (not a measured whole sweep)",
            "worldline_sweeps_per_s": 1.0 / per_wl,
            "sample": f"chain 0, first {k2} worldlines of each spin, 1 sweep ({dt2:.1f} s): "
                      f"{1.0 / per_wl:.3g} worldline-sweeps/s, divided by the {total_wl} worldlines of a "
                      f"whole {w['chains']}-chain sweep"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    w = WORK
    cores = oracle.num_threads()
    # one step = one sweep of a bounded sample (k worldlines per spin of chain 0)
    orc = oracle.Chain(w["L"], w["t"], w["U"], w["beta"], w["dtau"], w["filling"], 0)
    t0 = time.perf_counter()
    orc.sweep(nwl_limit=1)
    one = time.perf_counter() - t0
    budget = args.ref_seconds / max(1, args.steps + args.warmup)  # whole run within a few minutes
    k = max(1, min(orc.Nsig, int(budget / max(one, 1e-3) / 2)))
    for _ in range(args.warmup):
        orc.sweep(nwl_limit=k)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        orc.sweep(nwl_limit=k)
        times.append(time.perf_counter() - t0)
    per_wl = sum(times) / (len(times) * 2 * k)
    total_wl = w["chains"] * 2 * orc.Nsig
    value = 1.0 / (per_wl * total_wl)
    # a step is one sweep of the sample (2k worldlines of chain 0), which is what ms_per_step
    # measures; value is the per-worldline rate of those steps divided over the 65536
    # worldlines of a whole 64-chain sweep (the oracle cannot run a whole sweep in minutes)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "rate_kind": "per-worldline rate extrapolated from a sample: ms_per_step is one sweep of the sample, "
                         "value = 1 / (seconds per worldline-sweep x worldlines of a whole sweep)",
            "config": {"workload": WORKLOAD, "sample_worldlines_per_spin": k, "sample_chains": 1,
                       "worldlines_per_whole_sweep": total_wl},
            "cpu_baseline": {"value": value, "unit": "sweeps/s", "cores": cores, "kind": "oracle",
                             "worldline_sweeps_per_s": 1.0 / per_wl,
                             "sample": f"each step: chain 0, first {k} worldlines of each spin, one sweep; "
                                       f"per-worldline rate divided over {total_wl} worldlines"},
            "e2e": {"value": value, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


GRAD_WORKLOAD = ("adjoint: L=16 (N=256) t=1 U=4 beta=4 dtau=0.05 (M=80) half filling, 128 chains; "
                 "log Z, d log Z/d v and d log Z/d t per call, BF16 checkpoints every 9 slices")


def run_grad(args):
    """Adjoint evaluations per second (hqmc_log_weight_grad) on the L=16, 128-chain adjoint workload."""
    import numpy as np
    import torch

    from paper_2510_13866_gb300 import Lattice
    from paper_2510_13866_gb300.shard import chain_seeds

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    nch = args.chains or 128
    p = (1.0, 4.0, 4.0, 0.05, 1.0)
    lat = Lattice(16, chain_seeds(rank, nch), precision="fp32", device=local)
    lat.set_params(*p)
    lat.sweep(2)
    for _ in range(args.warmup):
        lat.log_weight_grad()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        lat.log_weight_grad()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    L, M, ns = lat.shapes[0]
    N = L * L
    part = nch * 2 * ns * M
    # forward, segment recompute and reverse pass (H and dG/dt * b): about four forward
    # filters of 5 N log2 N + 4 N flops per particle-slice
    flops = part * 4.0 * (5.0 * N * np.log2(N) + 4.0 * N)
    peak_alu, alu_src = alu_peak(local)
    cpu = None
    if not args.no_cpu and rank == 0:
        import oracle

        s, x, _, _ = lat.get_state(0)
        orc = oracle.Chain(16, *p, 0)
        orc.s[:] = s
        orc.x[:] = x
        t0 = time.perf_counter()
        orc.grad()
        dt = time.perf_counter() - t0
        cpu = {"value": 1.0 / (dt * nch), "unit": "gradient evaluations/s", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": f"chain 0 in full ({dt:.2f} s), extrapolated to {nch} chains"}
    lat.close()
    if rank == 0:
        line = {"metric": "gradient evaluations/s (log Z, d log Z/d v, d log Z/d t of every chain)",
                "value": world * 1e3 / ms, "unit": "evaluations/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": GRAD_WORKLOAD, "L": L, "M": M, "chains_per_gpu": nch},
                "roofline": {"bound": "alu", "achieved": flops / (ms / 1e3) / 1e12, "peak": peak_alu,
                             "unit": "TFLOP/s", "frac": flops / (ms / 1e3) / 1e12 / peak_alu, "traffic": None,
                             "kernel": "grad_kernel<float,16>", "peak_source": alu_src},
                "cpu_baseline": cpu, "gpu_launches": args.steps}
        print(json.dumps(line), flush=True)


WORKLOADS = {
    "L32": "the headline: " + WORKLOAD,
    "ragged": ("256 ragged chains, L in {8,12,16,24,32,48}, beta in {2,4,6}, U in {2,4,8}, filling in "
               "{0.5,0.875,1}, dtau=0.05, drawn per chain from Philox key (1,0); one graph replay per sweep"),
    "L64": "2D Hubbard L=64 (N=4096) t=1 U=4 beta=8 dtau=0.05 (M=160) half filling, 16 chains",
    "L128": "2D Hubbard L=128 (N=16384) t=1 U=4 beta=8 dtau=0.05 (M=160) half filling, 16 chains",
    "paper8": "the paper's regime: L=8, t=1, U=4, beta=32, dtau=1/32 (M=1024), half filling, 1 chain",
    "paper16": "the paper's regime: L=16, t=1, U=4, beta=32, dtau=1/32 (M=1024), half filling, 1 chain",
    "paper32": "the paper's regime: L=32, t=1, U=4, beta=32, dtau=1/32 (M=1024), half filling, 1 chain",
}


def workload(name, rank, chains, beta=None, U=None):
    """(L per chain, params per chain, seeds) of a named workload on rank `rank`."""
    from paper_2510_13866_gb300.shard import chain_seeds
    from paper_2510_13866_gb300.workloads import ragged

    if name == "L32":
        n = chains or WORK["chains"]
        p = (WORK["t"], WORK["U"], beta if beta else WORK["beta"], WORK["dtau"], WORK["filling"])
        return [32] * n, [p] * n, chain_seeds(rank, n)
    if name == "ragged":
        n = chains or 256
        work = ragged(n)
        return [w[0] for w in work], [w[1] for w in work], chain_seeds(rank, n)
    if name.startswith("paper"):
        L = int(name[5:])
        n = chains or 1
        return [L] * n, [(1.0, 4.0 if U is None else U, 32.0, 1.0 / 32.0, 1.0)] * n, chain_seeds(rank, n)
    L = int(name[1:])
    n = chains or 16
    return [L] * n, [(1.0, 4.0, beta if beta else 8.0, 0.05, 1.0)] * n, chain_seeds(rank, n)


def alu_peak(device):
    """(peak TFLOP/s, source): the measured packed-FP32 FMA rate of this GPU (the FFT
    kernels run packed f32x2), with the scalar FFMA rate and the nominal lane count beside it."""
    from paper_2510_13866_gb300 import fp32_peak

    _, _, sm_max = peaks()
    nominal = 152 * 128 * 2 * sm_max * 1e6 / 1e12
    try:
        packed, scalar = fp32_peak(device, True), fp32_peak(device, False)
    except Exception as e:  # noqa: BLE001 -- the roofline falls back to the nominal figure
        return nominal, f"nominal 152 SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz (probe failed: {e})"
    return packed, (f"measured in this run: packed f32x2 FMA loop {packed:.1f} TFLOP/s (scalar FFMA "
                    f"{scalar:.1f}; nominal 152 SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz = {nominal:.1f})")


def equilibrium_accuracy(obs32, obs64, burn, meas):
    """The FP32 filter against the plain FP64 form at equilibrium: independent chains of each
    precision (disjoint seeds) after `burn` sweeps, observables averaged over `meas` further
    sweeps per chain.  Per observable: both means with their statistical errors over the
    chains and z = (FP32 - FP64) / sqrt(se32^2 + se64^2); equal accuracy means |z| of order
    1 and standard errors of the same size."""
    import numpy as np

    names = ("double_occ", "m2", "ekin", "s_pipi", "density")
    a = np.array([[o[k] for k in names] for o in obs32])
    b = np.array([[o[k] for k in names] for o in obs64])
    sa = a.std(axis=0, ddof=1) / np.sqrt(len(a))
    sb = b.std(axis=0, ddof=1) / np.sqrt(len(b))
    out = {"burn_in_sweeps": burn, "measured_sweeps": meas, "chains_fp32": len(a), "chains_fp64": len(b),
           "seeds": "FP32 0..63, FP64 10000..10063 (disjoint)", "observables": {}}
    for j, k in enumerate(names):
        se = float(np.hypot(sa[j], sb[j]))
        d = float(a[:, j].mean() - b[:, j].mean())
        out["observables"][k] = {"fp32": float(a[:, j].mean()), "fp32_stat_err": float(sa[j]),
                                 "fp64": float(b[:, j].mean()), "fp64_stat_err": float(sb[j]),
                                 "z": d / se if se > 0 else None}
    zs = [v["z"] for v in out["observables"].values() if v["z"] is not None]
    out["max_abs_z"] = max(abs(z) for z in zs) if zs else None
    return out


def observables(lat, shapes, sweeps, open_path=True):
    """Observables of Sec. 4 after the timed region: the chains run `sweeps` more sweeps
    (with the open-path estimator on for n_k) and every estimate is the sign-reweighted
    mean over the chains, <O> = sum_c <sO>_c / sum_c <s>_c, with its standard error by the
    delta method over the independent chains.  S(k) and n_k are given along
    (0,0) -> (pi,0) -> (pi,pi) -> (0,0), C(r) along (r, 0) and the diagonal (r, r)."""
    import numpy as np

    L = shapes[0][0]
    if open_path:
        lat.set_measure_open(True)  # restarts the accumulators
    else:
        lat.measure(reset=True)
    lat.sweep(sweeps)
    obs = lat.measure()
    opn = lat.measure_open() if open_path else None
    sg = np.array([o["mean_sign"] for o in obs])
    n = len(sg)

    def est(vals):
        vals = np.asarray(vals, dtype=float)  # per chain (sign-reweighted within the chain)
        num = vals * sg.reshape((-1,) + (1,) * (vals.ndim - 1))
        R = num.mean(axis=0) / sg.mean()
        resid = num - R[None] * sg.reshape((-1,) + (1,) * (vals.ndim - 1))
        se = resid.std(axis=0, ddof=1) / np.sqrt(n) / abs(sg.mean()) if n > 1 else np.full(np.shape(R), np.nan)
        return R, se

    path = [(k, 0) for k in range(L // 2)] + [(L // 2, k) for k in range(L // 2)] + \
        [(k, k) for k in range(L // 2, -1, -1)]
    idx = [kx + L * ky for kx, ky in path]
    out = {"sweeps": sweeps, "chains": n,
           "mean_sign": {"value": float(sg.mean()), "stat_err": float(sg.std(ddof=1) / np.sqrt(n)) if n > 1 else None},
           "path": [[2 * kx / L, 2 * ky / L] for kx, ky in path], "path_unit": "pi"}
    for name in ("double_occ", "m2", "ekin", "s_pipi"):
        R, se = est([o[name] for o in obs])
        out[name] = {"value": float(R), "stat_err": float(se)}
    R, se = est([o["Sk"] for o in obs])
    out["Sk_path"] = {"value": R[idx].tolist(), "stat_err": se[idx].tolist()}
    R, se = est([o["Cr"] for o in obs])
    out["Cr_axis"] = {"value": R[:L // 2 + 1].tolist(), "stat_err": se[:L // 2 + 1].tolist()}
    dg = [r + L * r for r in range(L // 2 + 1)]
    out["Cr_diagonal"] = {"value": R[dg].tolist(), "stat_err": se[dg].tolist()}
    if opn is not None:
        R, se = est([nk for nk, _ in opn])
        out["nk_path"] = {"value": R[idx].tolist(), "stat_err": se[idx].tolist()}
    return out


def kernel_source_digest(workload="L32"):
    """Digest of the sources the workload's FFBS kernels compile from (the register kernel for
    L <= 32, the wide kernel too otherwise), comments and whitespace left out: the committed
    DRAM counters apply only to this code."""
    import hashlib
    import re

    h = hashlib.sha256()
    files = ("ffbs.cuh", "device_common.cuh") if workload == "L32" else ("ffbs.cuh", "ffbs_wide.cuh",
                                                                          "device_common.cuh")
    for f in files:
        with open(os.path.join(ROOT, "paper_2510_13866_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-seconds", type=float, default=150.0,
                    help="CPU seconds the reference arm (the oracle) spreads over its warm-up and timed steps")
    ap.add_argument("--fp64-steps", type=int, default=10,
                    help="timed sweeps of the plain FP64 form (taken at equilibrium, inside the accuracy run)")
    ap.add_argument("--acc-burn", type=int, default=100,
                    help="burn-in sweeps of the FP32 / FP64 equilibrium accuracy comparison (0: skip it)")
    ap.add_argument("--acc-sweeps", type=int, default=100,
                    help="measured sweeps per chain of the equilibrium accuracy comparison")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="L32", choices=sorted(WORKLOADS) + ["grad16"],
                    help="L32 (default, the headline configuration), ragged, L64, L128, paper8/16/32 "
                         "(M=1024); grad16 times the adjoint")
    ap.add_argument("--local-steps", type=int, default=20,
                    help="local-update sweeps timed beside the FFBS sweep (0: skip)")
    ap.add_argument("--fstore", default="stream", choices=["stream", "bf16", "f32"],
                    help="storage of f for the wide kernel's backward pass: every slice in FP32 (stream), or "
                         "checkpoints every ceil(sqrt M) slices in BF16 / FP32 with the segments recomputed")
    ap.add_argument("--conv", default="fft", choices=["fft", "stencil"],
                    help="line convolutions of the FFBS filter (stencil: the truncated-stencil comparison)")
    ap.add_argument("--perm", action="store_true",
                    help="permutation updates at tau = beta in every sweep (sign-reweighted observables)")
    ap.add_argument("--block", type=int, default=0,
                    help="FFBS block length B (0: the closed loop from the anchor, the default)")
    ap.add_argument("--slice-group", type=int, default=0,
                    help="slices per CTA of the Gibbs/measure kernel (0: the library's choice, the default)")
    ap.add_argument("--beta", type=float, default=None,
                    help="beta of the L64/L128 workloads (default 8; smaller only for profiling captures), "
                         "or of L32 in place of its beta = 4")
    ap.add_argument("--U", type=float, default=None,
                    help="U of the paper8/16/32 workloads (default 4; the paper's runs use 1 and 20)")
    ap.add_argument("--observables", type=int, default=0,
                    help="after the timed region, run this many measured sweeps and report the Sec. 4 "
                         "observables (mean sign, D, m2, E_kin, S(k), C(r), n_k) with errors over the chains")
    ap.add_argument("--chains", type=int, default=None,
                    help="chains per GPU (default: the workload's own; smaller only for profiling captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "grad16":
        return run_grad(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(v):
        if world == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64, device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    from paper_2510_13866_gb300 import Lattice

    Ls, pars, seeds = workload(args.workload, rank, args.chains, args.beta, args.U)
    nchains = len(Ls)

    def make(precision, seed_offset=0):
        lt = Lattice(Ls, [s + seed_offset for s in seeds], precision=precision, device=local)
        if len(set(pars)) == 1:
            lt.set_params(*pars[0])
        else:
            for c, p in enumerate(pars):
                lt.set_params(*p, chain=c)
        if args.block:
            lt.set_block(args.block)
        if args.slice_group:
            lt.set_slice_launch(args.slice_group)
        if args.perm:
            lt.set_permutations(True)
        if args.conv != "fft":
            lt.set_conv(args.conv)
        if args.fstore != "stream" and precision == "fp32":
            lt.set_ffbs_storage(args.fstore)
        lt.prepare()
        return lt

    lat = make("fp32")
    shapes = lat.shapes
    nclasses = len(set(Ls))
    stream = torch.cuda.current_stream(local)
    lat.sweep(args.warmup)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()

    clk_path = os.path.join(tempfile.gettempdir(), f"hqmc_clocks_{os.getpid()}.csv")
    proc, fh = start_clocks(clk_path)
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.sweep(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clocks = stop_clocks(proc, fh, clk_path, local)
    barrier()
    ms = max_over_ranks(ms)
    value = world * args.steps / (ms / 1e3)

    # FFBS kernel time from CUDA events around its launches on the launching streams
    # (same sweeps, plain launches)
    lat.set_profiling(args.steps)
    lat.sweep(args.steps)
    ffbs_ms, slice_ms, nprof = lat.profile_read()
    lat.set_profiling(0)
    ffbs_avg = ffbs_ms / max(1, nprof)
    slice_avg = slice_ms / max(1, nprof)
    # algorithmic work per launch: every particle-slice writes f_l (4N B) and reads it back
    # (4N B); 5 N log2 N + 4 N flops
    part_slices = sum(2 * ns * M for (_, M, ns) in shapes)
    alg_bytes = sum(2 * ns * M * 8.0 * L * L for (L, M, ns) in shapes)
    alg_flops = sum(2 * ns * M * (5.0 * L * L * np.log2(L * L) + 4.0 * L * L) for (L, M, ns) in shapes)
    ckpt_note = None
    if args.fstore != "stream" and max(Ls) > 32:
        # checkpoints every K = ceil(sqrt M) slices: f written and read back once per K slices
        # (2 bytes per site in BF16, 4 in FP32), and the filter run twice (forward, recompute);
        # the recomputed segment goes through a per-CTA buffer (written and read, FP32)
        cb = 2.0 if args.fstore == "bf16" else 4.0
        alg_bytes = sum(2 * ns * L * L * (2 * cb * np.ceil(M / np.ceil(np.sqrt(M))) + 8.0 * M) for (L, M, ns) in shapes)
        alg_flops *= 2.0
        ckpt_note = ("f kept every ceil(sqrt M) slices (" + args.fstore + "); bytes = checkpoints written and read + "
                     "the recomputed segments through the per-CTA buffer; flops = forward + recompute")
    hbm_peak, peak_src, sm_max = peaks()
    achieved = alg_bytes / (ffbs_avg / 1e3) / 1e9
    peak_alu, alu_src = alu_peak(local)
    achieved_flops = alg_flops / (ffbs_avg / 1e3) / 1e12
    traffic, traffic_note = None, "no committed DRAM counters for this workload"
    tp = os.path.join(ROOT, "profiles", "ffbs_traffic.json")
    if os.path.exists(tp):
        try:
            rec = json.load(open(tp)).get(args.workload)
            if rec and rec.get("kernel_digest") == kernel_source_digest(args.workload):
                traffic = rec["bytes_per_launch"] * (nchains / rec["chains"])
                traffic_note = rec["how"]
            elif rec:
                traffic_note = "kernel changed since the committed DRAM counters were taken"
        except Exception:
            traffic = None
    kname = {"L32": "ffbs_kernel<float,32>", "L64": "ffbs_wide_kernel<float,64>",
             "L128": "ffbs_wide_kernel<float,128>"}.get(args.workload, "FFBS launches (all sizes)")
    roofline = {"bound": "hbm" if ckpt_note is None else "alu", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic, "traffic_note": traffic_note,
                "peak_source": peak_src, "kernel": kname, "kernel_ms": ffbs_avg, "gibbs_measure_ms": slice_avg,
                "alg_bytes_per_launch": alg_bytes,
                "alu": {"achieved_tflops": achieved_flops, "peak_tflops": peak_alu,
                        "frac": achieved_flops / peak_alu, "peak_source": alu_src}}
    if ckpt_note is not None:
        # the recompute makes the checkpoint form an FP32-ALU-bound filter: the ALU figures
        # lead, the bytes stand beside them
        roofline.update({"achieved": achieved_flops, "peak": peak_alu, "unit": "TFLOP/s",
                         "frac": achieved_flops / peak_alu, "peak_source": alu_src, "traffic": None,
                         "traffic_note": "no DRAM counters for the checkpoint form",
                         "hbm": {"achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                                 "peak_source": peak_src},
                         "storage": ckpt_note})
    # the Gibbs/measure kernel: per site-slice two int32 counts read and cleared (16 B)
    # and the field bits written twice (2 x 1 bit); the counts were just written by the
    # FFBS atomics and sit in L2, so HBM is not what bounds it
    site_slices = sum(M * L * L for (L, M, _) in shapes)
    gibbs_bytes = site_slices * (16.0 + 0.25)
    roofline["gibbs"] = {"kernel": "slice_kernel", "kernel_ms": slice_avg, "alg_bytes_per_launch": gibbs_bytes,
                         "achieved": gibbs_bytes / (slice_avg / 1e3) / 1e9, "unit": "GB/s",
                         "frac_of_hbm": gibbs_bytes / (slice_avg / 1e3) / 1e9 / hbm_peak,
                         "note": "latency-bound: L2-resident counts, short CTAs"}

    # FP32 diagnostics over the sweeps run so far (degenerate draws are counted, not raised)
    obs = lat.measure(reset=True)
    n_sw = max(1, obs[0]["n_samples"])
    diag = {"degenerate_per_sweep": sum(o["n_degenerate"] for o in obs) / n_sw,
            "nonpositive_per_sweep": sum(o["n_nonpositive"] for o in obs) / n_sw,
            "draws_per_sweep": sum(2 * ns * (M - 1) for (_, M, ns) in shapes)}

    # end to end through the public API: host log-weight buffer every step
    ke = min(args.steps, 20)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        lat.sweep(1, logw=True)
    te = time.perf_counter() - t0
    e2e_val = max_over_ranks(te)
    e2e = {"value": world * ke / e2e_val, "unit": "sweeps/s", "h2d_bytes_per_step": 0,
           "d2h_bytes_per_step": int(8 * sum(2 * ns for (_, _, ns) in shapes)) + 4}
    phys = None
    if args.observables > 0 and nclasses == 1:
        phys = observables(lat, shapes, args.observables)
    # local link updates (Eq. Rlocal in the position basis) on the same chains: one
    # launch per slice colour, then the same Gibbs/measure step; plain launches
    local_upd = None
    if args.local_steps > 0:
        lat.measure(reset=True)
        lat.local_sweep(3)
        torch.cuda.synchronize()
        e0.record(stream)
        lat.local_sweep(args.local_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_loc = max_over_ranks(e0.elapsed_time(e1))
        nacc = sum(o["n_local_accepted"] for o in lat.measure(reset=True))
        proposals = (args.local_steps + 3) * sum(2 * ns * M for (_, M, ns) in shapes)
        local_upd = {"value": world * args.local_steps / (ms_loc / 1e3), "unit": "sweeps/s",
                     "steps": args.local_steps, "ms_per_sweep": ms_loc / args.local_steps,
                     "accepted_per_proposal": nacc / proposals, "launches_per_sweep": 5}
    lat.close()

    # plain FP64 form: same kernels in double, one launch per phase, no graph; timed at
    # equilibrium inside the accuracy comparison (disjoint seeds from the FP32 chains)
    fp64 = None
    if args.fp64_steps > 0 and max(Ls) <= 32:
        lat64 = make("fp64", seed_offset=10_000)
        burn = max(1, args.acc_burn)
        lat64.sweep(burn)
        lat64.measure(reset=True)
        torch.cuda.synchronize()
        e0.record(stream)
        lat64.sweep(args.fp64_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = max_over_ranks(e0.elapsed_time(e1))
        v64 = world * args.fp64_steps / (ms64 / 1e3)
        fp64 = {"value": v64, "unit": "sweeps/s", "steps": args.fp64_steps, "fp32_over_fp64": value / v64,
                "timed_after_sweeps": burn}
        # the FP64 form's own ALU roofline: the same algorithmic flops per sweep against
        # the measured DFMA rate (it runs the same FFTs in double)
        try:
            from paper_2510_13866_gb300 import fp64_peak

            p64 = fp64_peak(local)
            a64 = alg_flops / (ms64 / args.fp64_steps / 1e3) / 1e12
            fp64["alu"] = {"achieved_tflops": a64, "peak_tflops": p64, "frac": a64 / p64,
                           "peak_source": "measured in this run: DFMA loop on every SM"}
        except Exception as e:  # noqa: BLE001 -- the rate stands without its roofline
            fp64["alu"] = {"error": str(e)}
        if args.acc_burn > 0:
            try:
                lat64.sweep(max(0, args.acc_sweeps - args.fp64_steps))
                obs64 = lat64.measure()
                lat32 = make("fp32")
                lat32.sweep(burn)
                lat32.measure(reset=True)
                lat32.sweep(max(args.acc_sweeps, args.fp64_steps))
                obs32 = lat32.measure()
                lat32.close()
                fp64["accuracy"] = equilibrium_accuracy(obs32, obs64, burn, max(args.acc_sweeps, args.fp64_steps))
            except Exception as e:  # noqa: BLE001 -- an optional comparison; the line still prints
                fp64["accuracy"] = {"error": str(e)}
        lat64.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and args.workload == "L32":
        try:
            cpu = cpu_oracle_sample()
        except Exception as e:  # noqa: BLE001 -- the oracle is optional to the timed line
            cpu = {"error": str(e), "kind": "oracle"}

    if rank == 0:
        wl = WORKLOADS[args.workload]
        if args.workload == "L32" and nchains != WORK["chains"]:
            wl = wl.replace("x 64 chains", f"x {nchains} chains")
        if args.workload.startswith("paper") and nchains != 1:
            wl = wl.replace("1 chain", f"{nchains} chains")
        if args.workload.startswith("paper") and args.U is not None:
            wl = wl.replace("U=4", f"U={args.U:g}")
        if args.block:
            wl += f"; block FFBS, B={args.block}"
        if args.perm:
            wl += "; permutation updates at tau = beta"
        if args.conv != "fft":
            wl += "; line convolutions by the periodic stencil (|d| <= 6)"
        if args.fstore != "stream" and max(Ls) > 32:
            wl += f"; f checkpoints every ceil(sqrt M) slices in {args.fstore.upper()}, segments recomputed"
        if args.workload == "L32" and args.beta:
            wl += f"; beta={args.beta:g} instead (M={shapes[0][1]})"
        line = {"metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": wl, "L": sorted(set(Ls)) if nclasses > 1 else Ls[0],
                           "M": sorted(set(M for _, M, _ in shapes)) if nclasses > 1 else shapes[0][1],
                           "chains_per_gpu": nchains, "parallelism": f"chains sharded over {world} GPU(s)",
                           "l2": "per-sweep working set (f-message scratch, GBs) exceeds L2; no flush needed"
                           if not args.block else "FFBS blocks: the f-message working set is B slices per group"},
                "particle_slice_updates_per_s": value * part_slices,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": args.steps * (nclasses + 2 + (1 if args.perm else 0)), "clocks": clocks, "fp64_plain": fp64,
                "fp32_diagnostics": diag, "local_update": local_upd}
        if phys is not None:
            line["observables"] = phys
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
