"""Benchmark: Wilson-clover multigrid time-to-solution on one GB300 per rank.

The headline line is the largest single-GPU workload, 32^3x64 with three levels
(blocks 4^4 then 2^4: 8^3x16 and 4^3x8 coarse lattices, Nvec 24 / 32), FP32 inner
levels with BF16 coarse links (FP32 accumulation), FP64 outer FGMRES,
orthonormalisation and Hessenberg.  One step = one full pass of the hot path:
set the gauge field (clover term built on the device), the initial setup (the
near-null candidates drawn on the device by the seeded counter-based generator, 3
MR(4) sweeps per level), 2 iterative-refinement sweeps, and the FGMRES(20) solve of
D x = b to a true relative residual of 1e-10.  `value` is the time-to-solution in
seconds (device CUDA events on the call's stream, max over ranks), inputs resident
in HBM, L2 flushed (256 MiB write + 256 MiB read) between steps.  `e2e` is the
same step through the same C-ABI calls with pinned host buffers, copies included.

The other workloads ride on the same line as sub-records (a few timed steps each):
16^3x32 two-level (c2), 24^3x48 with 12 and 48 right-hand sides solved together and
an uneven batch of lattices in one graph launch (c4), and the learned coarse
correction trained on 16^3x32 and deployed on 32^3x64 (c5).  Each names its own
comparison with plain FP64 GPU multigrid on the same inputs.

Multi-GPU: the path does not shard (one lattice per GPU): N ranks run independent
replicas; the step time is the max over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3|c2|c4|c5|table2]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

WORKLOADS = {
    "c2": dict(workload="wilson-clover 2-level MG, 16^3x32, eps 0.25, m0 -0.2, csw 1.0, blocks 4^4 -> 4^3x8, "
                        "Nvec 24 (nbasis 48), 3 initial + 2 refinement sweeps, MR(4) smoother, GMRES(20) coarse to "
                        "0.05, FGMRES(20) to 1e-10, 1 Gaussian rhs",
               dims=(16, 16, 16, 32), eps=0.25, m0=-0.2, csw=1.0, blocks=[(4, 4, 4, 4)], nvec=[24],
               init_sweeps=3, refine_sweeps=2, gauge_seed=1002, source_seed=0, nrhs=1, links="f32"),
    "c3": dict(workload="wilson-clover 3-level MG, 32^3x64, eps 0.2, m0 -0.25, csw 1.0, blocks 4^4 -> 8^3x16 "
                        "-> 2^4 -> 4^3x8, Nvec 24 / 32 (nbasis 48 / 64), 3 initial + 2 refinement sweeps, MR(4) "
                        "smoother, GMRES(20) coarsest to 0.05, FGMRES(20) to 1e-10, 1 Gaussian rhs, FP32 inner "
                        "levels, BF16 coarse links (FP32 accumulation)",
               dims=(32, 32, 32, 64), eps=0.2, m0=-0.25, csw=1.0, blocks=[(4, 4, 4, 4), (2, 2, 2, 2)],
               nvec=[24, 32], init_sweeps=3, refine_sweeps=2, gauge_seed=1003, source_seed=0, nrhs=1,
               links="bf16"),
    "c4": dict(workload="wilson-clover 3-level MG, 24^3x48, eps 0.25, m0 -0.2, csw 1.0, blocks 4^4 -> 6^3x12 "
                        "-> 2^4 -> 3^3x6, Nvec 24 / 24 (nbasis 48), 3 initial + 2 refinement sweeps, "
                        "FGMRES(20) to 1e-10, NRHS Gaussian rhs solved together, BF16 coarse links (tcgen05 "
                        "multi-rhs coarse apply)",
               dims=(24, 24, 24, 48), eps=0.25, m0=-0.2, csw=1.0, blocks=[(4, 4, 4, 4), (2, 2, 2, 2)],
               nvec=[24, 24], init_sweeps=3, refine_sweeps=2, gauge_seed=1004, source_seed=0, nrhs=12,
               links="bf16"),
    "c5": dict(workload="learned coarse correction: PTC network trained on 16^3x32 (eps 0.25, m0 -0.2) on pairs "
                        "the multigrid generates (fresh pools, POOLS x 48 pairs), deployed unchanged on 32^3x64 (eps "
                        "0.25, m0 -0.2, blocks 4^4 -> 8^3x16, Nvec 24, 3 + 2 sweeps) in place of the coarse "
                        "correction, plain MG as fallback (ratio 0.9), FGMRES(20) to 1e-10, 1 Gaussian rhs",
               dims=(32, 32, 32, 64), eps=0.25, m0=-0.2, csw=1.0, blocks=[(4, 4, 4, 4)], nvec=[24], init_sweeps=3,
               refine_sweeps=2, gauge_seed=1005, source_seed=0, nrhs=1, learned_from="c2", links="f32",
               train=dict(npairs=48, batch=4, refresh=8, lr=1e-2, target_tol=1e-6, seed=5)),
    "table2": dict(workload="Table-2-shaped sweep: 16^4, eps 0.25, m0 -0.25, csw 1.0, blocks 4^4 -> 4^4, Nvec 20 "
                            "(nbasis 40), GMRES(4) smoother, 3 initial sweeps, 0..10 refinement sweeps, FGMRES(20) "
                            "to 1e-10, 1 Gaussian rhs",
                   dims=(16, 16, 16, 16), eps=0.25, m0=-0.25, csw=1.0, blocks=[(4, 4, 4, 4)], nvec=[20],
                   init_sweeps=3, refine_sweeps=0, gauge_seed=1006, source_seed=0, nrhs=1, smoother="gmres",
                   links="f32"),
}
DEFAULT_WORKLOAD = "c3"

# Operator applications of one step of the 32^3x64 workload (set_gauge, setup and
# the solve, host-driven), per kind and level, as the GPU arm's operator counters
# (wcmg_get_opcounts) recorded them; the GPU line carries its own live counts under
# cpu_baseline.  The reference arm multiplies the oracle's operator times by these.
OP_COUNTS = {"c3": {"apply": [892, 1180, 300, 0], "restrict": [108, 108, 0, 0], "prolong": [108, 108, 0, 0],
                    "ortho": [3, 3, 0, 0], "coarsen": [3, 3, 0, 0]}}

# DRAM traffic per launch of the dominant kernel from one ncu capture, valid only
# while the sources that define the kernel are unchanged (src_hash of its class).
NCU_TRAFFIC = {
    "dslash": {"bytes_per_launch": 14.42e9, "src": "dda1aff51ef44689",
               "how": "ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum "
                      "--clock-control none (one pass) over one 32^3x64 step (--graphs 0 --ncu-region): the 49 "
                      "fine-stencil launches of the set-up (20 + 2 Dslash with 24 rhs, 27 chirality-pair "
                      "stencils), 706.4 GB of DRAM traffic"},
}

KCLASS = ["dslash", "coarse", "restrict", "prolong", "blas", "ortho", "coarsen", "clover", "pack", "krylov",
          "dslash64", "other"]


# Sources that define each kernel class (its own file and the shared headers): a
# recorded ncu traffic figure stays valid while these files are unchanged.
KERNEL_SOURCES = {"ortho": ["transfer.cu", "dfloat.cuh"], "restrict": ["transfer.cu"], "prolong": ["transfer.cu"],
                  "dslash": ["fine.cu"], "dslash64": ["fine.cu"], "coarse": ["coarse.cu"], "blas": ["blas.cu"],
                  "krylov": ["blas.cu"], "coarsen": ["coarse.cu", "fine.cu"], "ptc": ["ptc.cu"]}


def src_hash(kernel_class=None) -> str:
    """sha256 prefix of the kernel class's sources (all CUDA sources when None)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1904_08678_gb300", "csrc")
    files = sorted(f for f in os.listdir(d) if f.endswith((".cu", ".cuh", ".h")))
    if kernel_class in KERNEL_SOURCES:
        files = sorted(KERNEL_SOURCES[kernel_class] + ["common.cuh"])
    for f in files:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), float(m["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


# FP64 / FP32 non-tensor ALU peaks of GB300 derived from unit counts and the
# maximum SM clock: 152 SMs x 2070 MHz x 2 flop/FMA x (2 FP64 / 128 FP32) FMA per SM per clock.
ALU_PEAK_TFLOPS = {"f64": 152 * 2.070e9 * 2 * 2 / 1e12, "f32": 152 * 2.070e9 * 2 * 128 / 1e12}


# ---------------------------------------------------------------- distributed
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend, init_method="env://")
    return dist


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device])
        else:
            dist.barrier()


def max_over_ranks(dist, value: float, device=None) -> float:
    """Max of a per-rank scalar over all ranks (identity at world size 1)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value: float, device=None) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------- clocks
def smi_id(local: int) -> str:
    """nvidia-smi identifier (GPU-<uuid>) of CUDA device `local`; its index if unknown."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(local).uuid)
        if u and u.lower() != "none":
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    return str(local)


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        # nvidia-smi numbers GPUs physically, CUDA within CUDA_VISIBLE_DEVICES: name the
        # device by its UUID so the samples come from the GPU this process runs on
        self.gpu = smi_id(gpu_index)
        self.proc = None
        # raw samples (the line carries their summary): BENCH_CLOCKS_DIR, else the temp dir
        d = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


class L2Flush:
    """Evict L2 (129 MB on GB300) between timed iterations: write a 256 MiB buffer, then read
    another 256 MiB buffer so the dirty lines are written back before the next timed kernel."""

    def __init__(self, torch, dev):
        self.w = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        self.r = torch.ones(64 << 20, dtype=torch.float32, device=dev)

    def fill_(self, v):
        self.w.fill_(v)
        self.sink = self.r.sum()


# ---------------------------------------------------------------- inputs
def level_dims(cfg):
    out = [tuple(cfg["dims"])]
    for b in cfg["blocks"]:
        out.append(tuple(L // x for L, x in zip(out[-1], b)))
    return out


def make_inputs(cfg, nrhs=None):
    """Gauge field and source(s) on the host.  The near-null candidates are drawn on
    the device from the gauge seed (wcmg_setup_seeded), so they are not made here."""
    from paper_1904_08678_gb300 import inputs
    dims = cfg["dims"]
    U = inputs.random_gauge(dims, cfg["eps"], cfg["gauge_seed"], workers=min(16, os.cpu_count() or 1))
    b = inputs.source(dims, cfg["source_seed"], nrhs=nrhs or cfg.get("nrhs", 1))
    return U, b


def params(wcmg, cfg, inner, links=None, profile=0, graphs=0, autotune=1, nrhs=None):
    links = links or cfg.get("links", "f32")
    ortho_df = int(cfg.get("ortho", "fp64") == "df" and inner == "f32")  # plain FP64 MG: FP64 throughout
    coarse_eo = int(cfg.get("coarse_eo", 0))
    sigma3 = int(cfg.get("sigma3", 0))
    p = wcmg.default_params(dims=cfg["dims"], blocks=cfg["blocks"], nvec=cfg["nvec"], m0=cfg["m0"], csw=cfg["csw"],
                            setup_init_sweeps=cfg["init_sweeps"], setup_refine_sweeps=cfg["refine_sweeps"],
                            n_levels=len(cfg["blocks"]) + 1, max_rhs=nrhs or cfg.get("nrhs", 1), profile=profile,
                            use_graphs=graphs, autotune=autotune,
                            smoother={"mr": wcmg.SMOOTHER_MR, "gmres": wcmg.SMOOTHER_GMRES,
                                      "sap": wcmg.SMOOTHER_SAP}[cfg.get("smoother", "mr")],
                            sap_cycles=int(cfg.get("sap_cycles", 1)), sap_eo=int(cfg.get("sap_eo", 0)),
                            smoother_steps=int(cfg.get("smoother_steps", 4)),
                            kcycle=int(cfg.get("kcycle", 0)), ortho_df=ortho_df, coarse_eo=coarse_eo,
                            coarse_sigma3=sigma3)
    p.inner_prec = {"f64": wcmg.F64, "f32": wcmg.F32}[inner]
    p.coarse_link_prec = {"f32": wcmg.F32, "bf16": wcmg.BF16, "f16": wcmg.F16}[links]
    return p


def add_stats(acc, st):
    for i in range(len(KCLASS)):
        k = st.k[i]
        a = acc.setdefault(KCLASS[i], [0, 0.0, 0.0, 0.0])
        a[0] += k.launches
        a[1] += k.ms
        a[2] += k.bytes
        a[3] += k.flops


def timed_call(torch, stream, flush, fn, tag=0):
    """One call of fn between CUDA events on `stream`, L2 flushed before; (result, ms)."""
    flush.fill_(tag & 0xFF)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    r = fn()
    b.record(stream)
    torch.cuda.synchronize()
    return r, a.elapsed_time(b)


# ---------------------------------------------------------------- GPU arm
class Env:
    """Per-process GPU context of the bench: torch, the binding, device, stream, L2 flush."""

    def __init__(self, local, dist, ncu_region=False):
        import torch
        from paper_1904_08678_gb300 import wcmg
        self.torch, self.wcmg, self.local, self.dist = torch, wcmg, local, dist
        self.ncu_region = ncu_region
        self.dev = torch.device("cuda", local)
        self.stream = torch.cuda.current_stream()
        self.flush = L2Flush(torch, self.dev)

    def to_dev(self, a):
        return self.torch.from_numpy(a).to(self.dev)


def opcount_delta(now, before):
    return {k: [a - b for a, b in zip(now[k], before[k])] for k in now}


def measure(env, cfg, steps, warmup, nrhs=None, inner="f32", graphs=1, autotune=1, e2e_steps=0, fp64=False,
            clocks=None, roofline=True, extra=None):
    """Time `steps` steps (set_gauge + seeded setup + solve) of workload cfg after
    `warmup` untimed ones.  The first warm-up step runs host-driven (the solve graph is
    captured on the second) and every kernel class is event-timed during the warm-up.
    The timed steps run with no per-launch timing; after them, up to two more steps
    time every launch of the dominant class for the roofline.  Returns the fields of a
    bench line (or sub-record)."""
    torch, wcmg, stream, flush = env.torch, env.wcmg, env.stream, env.flush
    nrhs = nrhs or cfg.get("nrhs", 1)
    U, b = make_inputs(cfg, nrhs)
    Ud, bd = env.to_dev(U), env.to_dev(b)
    xd = torch.zeros_like(bd)
    ctx = wcmg.Context(params(wcmg, cfg, inner, profile=-1, graphs=graphs, autotune=autotune, nrhs=nrhs))
    seed = cfg["gauge_seed"]

    def step(x, U_, b_):
        ctx.set_gauge(U_, stream)
        s1 = ctx.setup_seeded(seed, stream)
        s2 = ctx.solve(b_, x, nrhs=nrhs, stream=stream)
        return s1, s2

    acc, first_solve, opc = {}, None, None
    for i in range(warmup):
        oc0 = ctx.opcounts()
        flush.fill_(1)
        s1, s2 = step(xd, Ud, bd)
        add_stats(acc, s1)
        add_stats(acc, s2)
        if i == 0:
            first_solve, opc = s2, opcount_delta(ctx.opcounts(), oc0)
    torch.cuda.synchronize()
    warm_ms = {k: round(v[1] / warmup, 3) for k, v in acc.items() if v[1] > 0}
    dominant = max(acc, key=lambda k: acc[k][1])
    ctx.set_profile(0)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    acc = {}
    its, res, launches, coarse_its, graphs_used = [], [], 0, [], []
    phases = {"setup_init": [], "setup_refine": [], "solve": []}
    barrier(env.dist, env.local)
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    if clocks is not None:
        clocks.__enter__()
    if env.ncu_region:
        torch.cuda.profiler.start()  # ncu --profile-from-start off: profile the timed steps only
    try:
        for i in range(steps):
            flush.fill_(i & 0xFF)
            starts[i].record(stream)
            s1, s2 = step(xd, Ud, bd)
            ends[i].record(stream)
            add_stats(acc, s1)
            add_stats(acc, s2)
            its.append(s2.outer_iterations)
            graphs_used.append(s2.graph)
            coarse_its.append((s1.coarse_iterations, s2.coarse_iterations))
            res.append(s2.true_residual)
            launches += s1.kernel_launches + s2.kernel_launches + 2  # + set_gauge's pack/clover kernels
            phases["setup_init"].append(s1.ms_setup_init)
            phases["setup_refine"].append(s1.ms_setup_refine)
            phases["solve"].append(s2.ms_solve)
        torch.cuda.synchronize()
    finally:
        if env.ncu_region:
            torch.cuda.profiler.stop()
        if clocks is not None:
            clocks.__exit__(None, None, None)
    t_wall = time.perf_counter() - t_wall
    barrier(env.dist, env.local)
    step_ms = [starts[i].elapsed_time(ends[i]) for i in range(steps)]
    ms = max_over_ranks(env.dist, sum(step_ms) / len(step_ms), env.dev)
    med = lambda v: round(statistics.median(v), 2)
    out = {"time_to_solution_s": round(ms / 1e3, 5), "ms_per_step": round(ms, 3),
           "ms_each_step": [round(t, 3) for t in step_ms], "steps": steps, "warmup": warmup,
           "outer_iterations": its[-1], "true_residual": max(res), "phases_ms": {k: med(v) for k, v in phases.items()},
           "solve": "one CUDA graph per solve (device-side stopping tests)" if all(graphs_used) else "host-driven",
           "gpu_launches": launches, "gpu_launches_per_step": launches // steps,
           "coarse_gmres_iterations": {"setup": coarse_its[-1][0], "solve": coarse_its[-1][1]},
           "warmup_kernel_ms_per_step": warm_ms, "wall_s_timed": round(t_wall, 3), "op_counts": opc,
           "nrhs": nrhs, "inner_prec": inner, "coarse_links": cfg.get("links", "f32") if inner == "f32" else "f64"}

    if roofline:
        # the roofline pass: the dominant class's launches event-timed, outside the timed steps
        ctx.set_profile(1 << KCLASS.index(dominant))
        racc, rms, rsteps = {}, 0.0, min(2, steps)
        for i in range(rsteps):
            (s1, s2), t = timed_call(torch, stream, flush, lambda: step(xd, Ud, bd), i)
            add_stats(racc, s1)
            add_stats(racc, s2)
            rms += t
        ctx.set_profile(0)
        out["roofline"] = roofline_of(racc, dominant, rms / rsteps, rsteps, cfg.get("ortho") == "df")
    co = first_solve.k[KCLASS.index("coarse")]
    out["coarse_in_first_solve"] = {
        "launches": co.launches, "avg_launch_us": round(co.ms / max(co.launches, 1) * 1e3, 2),
        "GB/s": round(co.bytes / (co.ms * 1e-3) / 1e9, 1) if co.ms else None,
        "note": "host-driven first solve of the warm-up; links partly L2-resident between the applies of one "
                "coarse GMRES, so this is not an HBM fraction"}

    # launch shapes of the coarse applies (autotuned on first use, else the fixed rule)
    tiles = {}
    pr = wcmg.F64 if inner == "f64" else wcmg.F32
    for lev in range(1, len(cfg["blocks"]) + 1):
        for nr in sorted({1, nrhs, *cfg["nvec"]}):
            try:
                t = ctx.get_coarse_tile(lev, nr, pr)
            except wcmg.WcmgError:
                continue
            tiles[f"level{lev}_rhs{nr}"] = {k: (round(v, 2) if isinstance(v, float) else v) for k, v in t.items()}
    out["coarse_tiles"] = tiles

    if e2e_steps:
        Uh = torch.from_numpy(U).pin_memory()
        bh = torch.from_numpy(b).pin_memory()
        xh = torch.zeros_like(bh).pin_memory()
        e_ms = [timed_call(torch, stream, flush, lambda: step(xh, Uh, bh), 2)[1] for _ in range(e2e_steps)]
        e2e_ms = max_over_ranks(env.dist, sum(e_ms) / len(e_ms), env.dev)
        out["e2e"] = {"value": round(e2e_ms / 1e3, 5), "unit": "s", "h2d_bytes_per_step": U.nbytes + b.nbytes,
                      "d2h_bytes_per_step": b.nbytes, "steps": e2e_steps,
                      "note": "same step through the C-ABI with pinned host buffers: U and b copied in, x copied "
                              "out inside the timed region (the near-null candidates are drawn on the device)"}
    if fp64 and inner != "f64":
        out["fp64_inner"] = fp64_reference(env, cfg, Ud, bd, nrhs, graphs)
        out["fp64_inner"]["speedup_of_f32_inner"] = round(out["fp64_inner"]["time_to_solution_s"] * 1e3 / ms, 2)
    if extra is not None:
        extra(ctx, out, Ud, bd, xd, step)
    ctx.close()
    return out


# FP32 lane instructions per second of GB300: 152 SMs x 128 lanes x 2070 MHz.
FP32_INSTR_PEAK_T = 152 * 128 * 2.070e9 / 1e12
# FP32 instructions of one double-float real multiply-add (1 FMUL, 3 FFMA, 8 FADD)
DF_INSTR_PER_MAC = 12


def roofline_of(acc, dominant, ms, steps, ortho_df=False):
    hbm, bf16, peak_kind = peaks()
    d = acc[dominant]
    bound = "alu" if dominant in ("dslash64", "ortho") else "hbm"
    if bound == "hbm":
        achieved, peak, unit = d[2] / (d[1] * 1e-3) / 1e9, hbm, "GB/s"
        src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if peak_kind == "measured" else "fallback 6.8 TB/s"
    elif dominant == "ortho" and ortho_df:
        # double-float on the FP32 pipe: the algorithmic real multiply-adds of one
        # Gram-Schmidt pass (flops / 2), 12 FP32 instructions each
        achieved = d[3] / 2 * DF_INSTR_PER_MAC / (d[1] * 1e-3) / 1e12
        peak, unit = FP32_INSTR_PEAK_T, "T FP32 instructions/s"
        src = ("FP32 lanes x max SM clock (derived: 152 x 128 x 2.07 GHz); algorithmic work = one Gram-Schmidt "
               "pass in double-float, 12 FP32 instructions per real multiply-add")
    else:
        achieved, peak, unit = d[3] / (d[1] * 1e-3) / 1e12, ALU_PEAK_TFLOPS["f64"], "TFLOP/s"
        src = "FP64 unit count x max SM clock (derived; a DFMA probe measured 1.20 TFLOP/s at 1.99 GHz)"
    tr = NCU_TRAFFIC.get(dominant)
    traffic = tr["bytes_per_launch"] if tr and tr["src"] == src_hash(dominant) else None
    return {"kernel": dominant, "bound": bound, "achieved": round(achieved, 3), "peak": peak, "unit": unit,
            "frac": round(achieved / peak, 4), "peak_source": src, "traffic": traffic,
            "traffic_source": tr.get("how") if traffic is not None else None,
            "launches": d[0], "avg_launch_us": round(d[1] / max(d[0], 1) * 1e3, 2),
            "algorithmic_bytes_per_launch": d[2] / max(d[0], 1), "algorithmic_flops_per_launch": d[3] / max(d[0], 1),
            "share_of_step": round(d[1] / (ms * steps), 4),
            "timing": f"CUDA-event pair around every launch of this class (the library's stream) in {steps} extra "
                      "step(s) after the timed ones; the timed steps carry no per-launch events"}


def fp64_reference(env, cfg, Ud, bd, nrhs, graphs=1):
    """Plain FP64 GPU multigrid (same field, source and seeded setup): one timed step
    after a warm-up (setup, then two solves: host-driven and the graph capture)."""
    torch, wcmg, stream = env.torch, env.wcmg, env.stream
    c = wcmg.Context(params(wcmg, cfg, "f64", profile=0, graphs=graphs, nrhs=nrhs))
    x = torch.zeros_like(bd)
    c.set_gauge(Ud, stream)
    c.setup_seeded(cfg["gauge_seed"], stream)
    for _ in range(2):
        c.solve(bd, x, nrhs=nrhs, stream=stream)

    def run():
        c.set_gauge(Ud, stream)
        s1 = c.setup_seeded(cfg["gauge_seed"], stream)
        return s1, c.solve(bd, x, nrhs=nrhs, stream=stream)

    (s1, s2), ms = timed_call(torch, stream, env.flush, run, 3)
    c.close()
    return {"time_to_solution_s": round(ms / 1e3, 4), "outer_iterations": s2.outer_iterations,
            "true_residual": s2.true_residual, "setup_init_ms": round(s1.ms_setup_init, 2),
            "setup_refine_ms": round(s1.ms_setup_refine, 2), "solve_ms": round(s2.ms_solve, 2), "steps": 1}


def run_gpu(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    env = Env(local, dist, args.ncu_region)
    wcmg = env.wcmg
    name = args.workload
    cfg = dict(WORKLOADS[name])
    if args.links:
        cfg["links"] = args.links
    cfg["ortho"] = args.ortho
    if args.coarse_eo:
        cfg["coarse_eo"] = 1
        cfg["workload"] = cfg["workload"] + ", even-odd preconditioned coarsest solve"
    if args.sigma3:
        cfg["sigma3"] = 1
        cfg["workload"] = cfg["workload"] + ", five-block (sigma3) coarse-link copies available to the autotuner"
    if args.kcycle:
        cfg["kcycle"] = 1
        cfg["workload"] = cfg["workload"] + ", K-cycle (FGMRES(5) to 0.1 on the intermediate levels)"
    if args.smoother != "mr" or args.smoother_steps != 4:
        k = args.smoother_steps
        cfg["smoother"] = args.smoother
        cfg["sap_cycles"] = args.sap_cycles
        cfg["smoother_steps"] = k
        cfg["sap_eo"] = int(args.sap_eo)
        eo = ", even-odd preconditioned" if args.sap_eo else ""
        desc = {"mr": f"MR({k}) smoother", "gmres": f"GMRES({k}) smoother",
                "sap": f"SAP smoother ({args.sap_cycles} cycle(s) over the aggregates, MR({k}) per block{eo})"}[
            args.smoother]
        w = cfg["workload"]
        cfg["workload"] = w.replace("MR(4) smoother", desc) if "MR(4) smoother" in w else w + ", " + desc
    nrhs = args.nrhs or cfg.get("nrhs", 1)
    clk = ClockSampler(local)
    hbm = peaks()[0]

    def extra_main(ctx, out, Ud, bd, xd, step):
        out["near_null_quality"] = near_null_quality(env, ctx, cfg)
        refs = link_contexts(env, cfg)
        try:
            out["precision_per_level"] = precision_per_level(env, ctx, cfg, refs)
            out["coarse_stencil"] = coarse_isolated_levels(env, ctx, cfg, hbm, refs)
        finally:
            for c in refs.values():
                c.close()

    main = measure(env, cfg, args.steps, args.warmup, nrhs=nrhs, inner=args.inner, graphs=args.graphs,
                   autotune=args.autotune, e2e_steps=min(args.steps, 5),
                   fp64=(args.inner == "f32" and not args.no_fp64_compare), clocks=clk, extra=extra_main)
    ms = main["ms_per_step"]
    env.ncu_region = False  # only the headline's timed steps are bracketed
    sub = None
    if name == DEFAULT_WORKLOAD and not args.no_sub:
        sub = sub_records(env, args)
    elif name == "c2" and not args.no_learned:
        main["learned"] = learned_variant(env, cfg, args)
    elif name == "c4":
        main["uneven_batch"] = measure_uneven_batch(env, args)
    elif name == "c5":
        main["learned"] = learned_c5(env, cfg, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and name == DEFAULT_WORKLOAD:
        cpu = oracle_model(main["op_counts"], cfg)
        one = oracle_model_one_core(main["op_counts"], name)
        if one is not None:
            cpu["one_core"] = one

    if rank == 0:
        line = {
            "metric": "time_to_solution_1e-10", "value": main["time_to_solution_s"], "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "ms_each_step": main["ms_each_step"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.inner == "f32" else "f64", "data": "synthetic",
            "config": {"workload": cfg["workload"].replace("NRHS", str(nrhs)), "dims": list(cfg["dims"]),
                       "nrhs": nrhs, "inner_prec": args.inner, "solve": main["solve"],
                       "coarse_links": main["coarse_links"],
                       "l2": "flushed between steps (256 MiB write + 256 MiB read)", "parallelism": f"replicas x{world}",
                       "gauge": f"U = exp(i eps X), X = sum_a xi_a lambda_a, seed {cfg['gauge_seed']}",
                       "setup_vectors": "drawn on the device from the gauge seed (wcmg_setup_seeded)"},
            "outer_iterations": main["outer_iterations"], "true_residual": main["true_residual"],
            "phases_ms": main["phases_ms"],
            "solves_per_s": round(sum_over_ranks(dist, args.steps, env.dev) / (ms * args.steps / 1e3), 4),
            "roofline": main["roofline"], "coarse_stencil": main.get("coarse_stencil"),
            "coarse_in_first_solve": main["coarse_in_first_solve"],
            "e2e": main.get("e2e"), "fp64_inner": main.get("fp64_inner"),
            "precision_per_level": main.get("precision_per_level"),
            "learned": main.get("learned"), "uneven_batch": main.get("uneven_batch"),
            "coarse_tiles": main["coarse_tiles"], "op_counts": main["op_counts"],
            "gpu_launches": main["gpu_launches"], "gpu_launches_per_step": main["gpu_launches_per_step"],
            "clocks": clk.summary(), "wall_s_timed": main["wall_s_timed"], "cpu_baseline": cpu,
            "warmup_kernel_ms_per_step": main["warmup_kernel_ms_per_step"],
            "coarse_gmres_iterations": main["coarse_gmres_iterations"],
            "near_null_quality": main.get("near_null_quality"),
            "sub_records": sub,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def sub_records(env, args):
    """The other workloads, a few timed steps each (3 warm-up steps, --sub-steps timed)."""
    k = args.sub_steps
    out = {}
    c2 = dict(WORKLOADS["c2"], ortho=args.ortho)
    r = measure(env, c2, k, 3, e2e_steps=k, fp64=True, roofline=False)
    r["workload"] = c2["workload"]
    r["learned"] = learned_variant(env, c2, args)
    out["c2"] = r
    c4 = dict(WORKLOADS["c4"], ortho=args.ortho)
    out["c4"] = {"workload": c4["workload"].replace("NRHS", "12 or 48")}
    for nr in (12, 48):
        out["c4"][f"rhs{nr}"] = measure(env, c4, k, 3, nrhs=nr, fp64=(nr == 12), roofline=False)
    out["c4"]["uneven_batch"] = measure_uneven_batch(env, args)
    c5 = dict(WORKLOADS["c5"], ortho=args.ortho)
    out["c5"] = {"workload": c5["workload"].replace("POOLS", str(args.pools))}
    out["c5"].update(learned_c5(env, c5, args))
    return out


def learned_variant(env, cfg, args):
    """Learned coarse correction on the same field: train the PTC network on 24 pairs the
    multigrid generates, then time setup + solve with the network replacing the coarse
    correction (fallback ratio 0.9) and as a warm start of the coarsest GMRES."""
    torch, wcmg, stream, flush = env.torch, env.wcmg, env.stream, env.flush
    ctx = wcmg.Context(params(wcmg, cfg, "f32", profile=0))
    U, b = make_inputs(cfg)
    Ud, bd = env.to_dev(U), env.to_dev(b)
    seed = cfg["gauge_seed"]
    out = {}
    ctx.set_gauge(Ud, stream)
    ctx.setup_seeded(seed, stream)
    tr, ms_train = timed_call(torch, stream, flush, lambda: ctx.ptc_train(npairs=24, batch=4, steps=300, lr=1e-2,
                                                                         target_tol=1e-6, seed=5, stream=stream), 7)
    out["train"] = {"pairs": 24, "steps": 300, "batch": 4, "loss_initial": round(tr.loss_initial, 4),
                    "loss_final": round(tr.loss_final, 4), "ms": round(ms_train, 1),
                    "ms_generate": round(tr.ms_generate, 1)}
    for name, mode in (("plain_mg", wcmg.COARSE_MG), ("learned_replace", wcmg.COARSE_LEARNED),
                       ("learned_warmstart", wcmg.COARSE_WARMSTART)):
        ctx.set_coarse_mode(mode, 0.9)
        x = torch.zeros_like(bd)

        def run():
            ctx.set_gauge(Ud, stream)
            ctx.setup_seeded(seed, stream)
            return ctx.solve(bd, x, stream=stream)

        run()  # warm
        st, ms = timed_call(torch, stream, flush, run, 7)
        out[name] = {"time_to_solution_s": round(ms / 1e3, 5), "outer_iterations": st.outer_iterations,
                     "coarse_iterations": st.coarse_iterations, "solve_ms": round(st.ms_solve, 2),
                     "true_residual": st.true_residual, "learned_cycles": st.learned_cycles,
                     "fallback": st.learned_fallback}
    ctx.close()
    return out


def learned_c5(env, cfg, args, reps=3):
    """Configuration 5: train the PTC network on the 16^3x32 workload (pairs from its own
    multigrid, a fresh pool of 48 every 8 steps), deploy it unchanged on 32^3x64 in
    place of the coarse correction and as a warm start of the coarsest GMRES, against
    plain FP32 and FP64 multigrid on the same field, source and seeded setup."""
    torch, wcmg, stream, flush = env.torch, env.wcmg, env.stream, env.flush
    src = dict(WORKLOADS[cfg["learned_from"]], ortho=cfg.get("ortho", "fp64"))
    tr = dict(cfg["train"])
    Us, _ = make_inputs(src)
    c = wcmg.Context(params(wcmg, src, "f32", profile=0))
    c.set_gauge(env.to_dev(Us), stream)
    c.setup_seeded(src["gauge_seed"], stream)
    steps = args.pools * tr["refresh"]
    t0 = time.perf_counter()
    st = c.ptc_train(npairs=tr["npairs"], batch=tr["batch"], steps=steps, lr=tr["lr"], target_tol=tr["target_tol"],
                     seed=tr["seed"], refresh=tr["refresh"], stream=stream)
    wall = time.perf_counter() - t0
    W = torch.zeros(3456, dtype=torch.complex128, device=env.dev)
    c.ptc_get_weights(W, stream)
    c.close()
    out = {"trained_on": src["workload"], "pairs_total": st.pairs_total, "steps": steps, "batch": tr["batch"],
           "loss_initial": round(st.loss_initial, 4), "loss_final": round(st.loss_final, 4),
           "loss_heldout": round(st.loss_heldout, 4), "ms_generate": round(st.ms_generate, 1),
           "ms_train": round(st.ms_train, 1), "train_wall_s": round(wall, 2)}
    U, b = make_inputs(cfg)
    Ud, bd = env.to_dev(U), env.to_dev(b)
    xd = torch.zeros_like(bd)
    ctx = wcmg.Context(params(wcmg, cfg, "f32", profile=0, graphs=1))
    ctx.ptc_set_weights(W, stream)
    seed = cfg["gauge_seed"]

    def step():
        ctx.set_gauge(Ud, stream)
        s1 = ctx.setup_seeded(seed, stream)
        return s1, ctx.solve(bd, xd, stream=stream)

    dep = {}
    for name, mode in (("learned_replace", wcmg.COARSE_LEARNED), ("learned_warmstart", wcmg.COARSE_WARMSTART),
                       ("plain_mg", wcmg.COARSE_MG)):
        ctx.set_coarse_mode(mode, 0.9)
        step()
        step()  # warm (and, for plain MG, the graph capture)
        ms = []
        for i in range(reps):
            (s1, s2), t = timed_call(torch, stream, flush, step, i)
            ms.append(t)
        dep[name] = {"time_to_solution_s": round(statistics.median(ms) / 1e3, 5), "steps": reps,
                     "outer_iterations": s2.outer_iterations, "coarse_iterations": s2.coarse_iterations,
                     "solve_ms": round(s2.ms_solve, 2), "true_residual": s2.true_residual,
                     "learned_cycles": s2.learned_cycles, "fallback": s2.learned_fallback, "graph": s2.graph}
    ctx.close()
    dep["fp64_plain_mg"] = fp64_reference(env, cfg, Ud, bd, 1)
    out["deployed"] = dep
    return out


def link_contexts(env, cfg):
    """Contexts of the workload's geometry whose coarse links are set from another
    context: one per link storage (FP64 with FP64 applies; FP32, BF16, FP16 with FP32)."""
    wcmg = env.wcmg
    return {lp: wcmg.Context(params(wcmg, cfg, "f64" if lp == "f64" else "f32", "f32" if lp == "f64" else lp,
                                    profile=0, autotune=0)) for lp in ("f32", "bf16", "f16", "f64")}


def precision_per_level(env, ctx, cfg, refs):
    """Error of each level's FP32 transfers and of the coarse apply in FP32 / BF16 / FP16
    link storage, each against the FP64 apply of the same operator (the level's links as
    this setup built them, applied by an FP64 context), on a Gaussian vector."""
    torch, wcmg, stream = env.torch, env.wcmg, env.stream
    from paper_1904_08678_gb300 import inputs
    ld = level_dims(cfg)
    nl = len(cfg["blocks"]) + 1
    out = {}

    def rel(a, b):
        return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))

    for l in range(1, nl):
        Vc = int(np.prod(ld[l]))
        nb = 2 * cfg["nvec"][l - 1]
        A = torch.zeros((9, Vc, nb, nb), dtype=torch.complex128, device=env.dev)
        ctx.get_coarse_links(l, A, stream)
        x = env.to_dev(inputs.complex_gaussian(77, l, (1, Vc, nb)))
        y = {}
        for lp, c in refs.items():
            c.set_coarse_links(l, A, stream)
            y[lp] = torch.zeros_like(x)
            c.apply_coarse(l, x, y[lp], nrhs=1, prec=wcmg.F64 if lp == "f64" else wcmg.F32, stream=stream)
        Vf = int(np.prod(ld[l - 1]))
        nf = 12 if l == 1 else 2 * cfg["nvec"][l - 2]
        f = env.to_dev(inputs.complex_gaussian(78, l, (1, Vf, nf)))
        r64, r32 = torch.zeros_like(x), torch.zeros_like(x)
        ctx.restrict(l - 1, f, r64, prec=wcmg.F64, stream=stream)
        ctx.restrict(l - 1, f, r32, prec=wcmg.F32, stream=stream)
        p64, p32 = torch.zeros_like(f), torch.zeros_like(f)
        ctx.prolong(l - 1, x, p64, prec=wcmg.F64, stream=stream)
        ctx.prolong(l - 1, x, p32, prec=wcmg.F32, stream=stream)
        out[f"level{l}"] = {"coarse_apply_f32": rel(y["f32"], y["f64"]), "coarse_apply_bf16": rel(y["bf16"], y["f64"]),
                            "coarse_apply_f16": rel(y["f16"], y["f64"]), "restrict_f32": rel(r32, r64),
                            "prolong_f32": rel(p32, p64), "sites": Vc, "nbasis": nb}
    out["note"] = ("relative error ||y - y64|| / ||y64|| of one application on a Gaussian vector; y64 = the FP64 "
                   "apply of the same (FP32-built) coarse links and FP64 near-null vectors")
    return out


def near_null_quality(env, ctx, cfg):
    """How near-null the setup's vectors are: ||D_l v_i|| / ||v_i|| for each near-null
    vector of every level that has them (level 0 with the FP64 D, coarser levels with the
    level's coarse operator in FP32 arithmetic), next to the same ratio for a Gaussian
    vector.  Small ratios mean a good coarse space."""
    torch, wcmg, stream = env.torch, env.wcmg, env.stream
    from paper_1904_08678_gb300 import inputs
    ld = level_dims(cfg)
    out = {}
    for l in range(len(cfg["blocks"])):
        V = int(np.prod(ld[l]))
        nc = 12 if l == 0 else 2 * cfg["nvec"][l - 1]
        nv = cfg["nvec"][l]
        vecs = torch.zeros((nv, V, nc), dtype=torch.complex128, device=env.dev)
        ctx.get_nullvecs(l, vecs, stream)
        y = torch.zeros((1, V, nc), dtype=torch.complex128, device=env.dev)

        def ratio(v):
            if l == 0:
                ctx.apply_D(v, y, nrhs=1, prec=wcmg.F64, stream=stream)
            else:
                ctx.apply_coarse(l, v, y, nrhs=1, prec=wcmg.F32, stream=stream)
            return float(torch.linalg.vector_norm(y) / torch.linalg.vector_norm(v))

        r = [ratio(vecs[i:i + 1].contiguous()) for i in range(nv)]
        g = ratio(env.to_dev(inputs.complex_gaussian(79, l, (1, V, nc))))
        out[f"level{l}"] = {"mean": round(float(np.mean(r)), 4), "min": round(min(r), 4), "max": round(max(r), 4),
                            "gaussian_vector": round(g, 4), "vectors": nv}
        del vecs
    out["note"] = "||D_l v|| / ||v|| of the near-null vectors after the setup (3 + 2 sweeps)"
    return out


def coarse_isolated_levels(env, ctx, cfg, hbm, refs, reps=200):
    """K4 alone, 1 rhs, L2 flushed before every apply, on every coarse level of the
    workload with the links this setup built, stored as FP64, FP32 and the workload's
    BF16 / FP16 (FP32 vectors): time per apply and GB/s of the algorithmic bytes
    V_c (9 nb^2 s_link + 2 nb s_vec).  Level 1 is also compared with a device copy of
    the same byte count timed the same way."""
    torch, wcmg, stream, flush = env.torch, env.wcmg, env.stream, env.flush
    from paper_1904_08678_gb300 import inputs
    ld = level_dims(cfg)
    out = {}
    stores = [("f64", wcmg.F64, 16, 16), ("f32", wcmg.F32, 8, 8)]
    if cfg.get("links", "f32") in ("bf16", "f16"):
        stores.append((cfg["links"], wcmg.F32, 4, 8))
    ctxs = refs
    for c in ctxs.values():
        c.set_profile(1 << KCLASS.index("coarse"))
    for l in range(1, len(cfg["blocks"]) + 1):
        Vc = int(np.prod(ld[l]))
        nb = 2 * cfg["nvec"][l - 1]
        A = torch.zeros((9, Vc, nb, nb), dtype=torch.complex128, device=env.dev)
        ctx.get_coarse_links(l, A, stream)
        phi = env.to_dev(inputs.complex_gaussian(5, 5, (1, Vc, nb)))
        y = torch.zeros_like(phi)
        lev = {"sites": Vc, "nbasis": nb}
        for name, prec, link_b, vec_b in stores:
            c = ctxs[name]
            c.set_coarse_links(l, A, stream)
            algo = Vc * (9 * nb * nb * link_b + 2 * nb * vec_b)
            for _ in range(5):
                c.apply_coarse(l, phi, y, prec=prec, stream=stream)  # autotune, warm
            c.tune_coarse(l, 1, prec, cold=1, stream=stream)
            k0 = c.kstats()["coarse"]
            for _ in range(reps):
                flush.fill_(5)
                c.apply_coarse(l, phi, y, prec=prec, stream=stream)
            torch.cuda.synchronize()
            k1 = c.kstats()["coarse"]
            n = k1["launches"] - k0["launches"]
            kms = (k1["ms"] - k0["ms"]) / max(n, 1)
            t = c.get_coarse_tile(l, 1, prec)
            lev[f"links_{name}"] = {"link_bytes": link_b, "vector_bytes": vec_b, "algorithmic_bytes": algo,
                                    "kernel_us": round(kms * 1e3, 2), "GB/s": round(algo / (kms * 1e-3) / 1e9, 1),
                                    "frac_of_hbm": round(algo / (kms * 1e-3) / 1e9 / hbm, 4), "applies": n,
                                    "tile": {k: t[k] for k in ("kind", "rhs_per_cta", "parts", "threads", "ntile")}}
        out[f"level{l}"] = lev
    for c in ctxs.values():
        c.set_profile(0)
    # context for the ratio: the measured HBM peak is a 2 GiB + 2 GiB copy; a device copy
    # moving the level-1 apply's bytes (half read, half written), timed the same way
    lk = cfg.get("links", "f32") if cfg.get("links", "f32") in ("bf16", "f16") else "f32"
    algo = out["level1"][f"links_{lk}"]["algorithmic_bytes"]
    src = torch.empty(algo // 2, dtype=torch.uint8, device=env.dev)
    dst = torch.empty_like(src)
    times = []
    for i in range(60):
        _, t = timed_call(torch, stream, flush, lambda: dst.copy_(src), 6)
        if i >= 10:
            times.append(t * 1e3)
    copy_us = float(np.median(times))
    copy_gbs = 2 * (algo // 2) / (copy_us * 1e-6) / 1e9
    out["level1"]["same_size_copy"] = {"bytes": 2 * (algo // 2), "us": round(copy_us, 2), "GB/s": round(copy_gbs, 1),
                                       "frac_of_hbm": round(copy_gbs / hbm, 4),
                                       "apply_frac_of_copy": round(out["level1"][f"links_{lk}"]["GB/s"] / copy_gbs, 4),
                                       "links": lk}
    if cfg.get("sigma3"):
        five_block_isolated(env, ctx, cfg, hbm, out, reps)
    out["l2"] = "flushed before every apply (256 MiB write + 256 MiB read); launch shape from the cold autotuner"
    return out


def five_block_isolated(env, ctx, cfg, hbm, out, reps):
    """The one-rhs apply from the five-block storage (launch kind 5) on the workload's own
    Galerkin links (the headline context, its link storage, FP32 vectors), L2 flushed
    before every apply: the fastest of its launch shapes, with GB/s of its own bytes
    V_c (5 nb^2 s_link + 2 nb s_vec) and of the nine-block bytes of the same apply."""
    torch, wcmg, stream, flush = env.torch, env.wcmg, env.stream, env.flush
    from paper_1904_08678_gb300 import inputs
    ld = level_dims(cfg)
    lk = cfg.get("links", "f32")
    link_b = {"f32": 8, "bf16": 4, "f16": 4}[lk]
    ctx.set_profile(1 << KCLASS.index("coarse"))
    try:
        for l in range(1, len(cfg["blocks"]) + 1):
            Vc = int(np.prod(ld[l]))
            nb = 2 * cfg["nvec"][l - 1]
            phi = env.to_dev(inputs.complex_gaussian(5, 5, (1, Vc, nb)))
            y = torch.zeros_like(phi)
            saved = ctx.get_coarse_tile(l, 1, wcmg.F32)

            def time_apply(n):
                k0 = ctx.kstats()["coarse"]
                for _ in range(n):
                    flush.fill_(5)
                    ctx.apply_coarse(l, phi, y, prec=wcmg.F32, stream=stream)
                torch.cuda.synchronize()
                k1 = ctx.kstats()["coarse"]
                return (k1["ms"] - k0["ms"]) / max(k1["launches"] - k0["launches"], 1)

            best = None
            for th in (128, 256, 512):
                for stg in (1, 2):
                    ctx.set_coarse_tile(l, 1, wcmg.F32, kind=5, threads=th, parts=1, stages=stg)
                    time_apply(3)
                    kms = time_apply(20)
                    if best is None or kms < best[0]:
                        best = (kms, dict(threads=th, parts=1, stages=stg))
            ctx.set_coarse_tile(l, 1, wcmg.F32, kind=5, **best[1])
            kms = time_apply(reps)
            algo5 = Vc * (5 * nb * nb * link_b + 2 * nb * 8)
            algo9 = Vc * (9 * nb * nb * link_b + 2 * nb * 8)
            out[f"level{l}"][f"links_{lk}_five_block"] = {
                "link_bytes": link_b, "vector_bytes": 8, "algorithmic_bytes": algo5,
                "kernel_us": round(kms * 1e3, 2), "GB/s": round(algo5 / (kms * 1e-3) / 1e9, 1),
                "frac_of_hbm": round(algo5 / (kms * 1e-3) / 1e9 / hbm, 4),
                "nine_block_equivalent_frac": round(algo9 / (kms * 1e-3) / 1e9 / hbm, 4),
                "tile": dict(kind=5, **best[1]), "applies": reps}
            # back to the shape the headline used
            if saved.get("source") == 2:
                ctx.set_coarse_tile(l, 1, wcmg.F32, kind=saved["kind"], rhs_per_cta=saved["rhs_per_cta"],
                                    parts=saved["parts"], threads=saved["threads"], ntile=saved["ntile"],
                                    stages=saved["stages"])
            else:
                ctx.set_coarse_tile(l, 1, wcmg.F32, kind=-1)
    finally:
        ctx.set_profile(0)


UNEVEN_BATCH = dict(
    lattices=[(8, 8, 8, 8), (12, 12, 12, 24), (16, 16, 16, 32)], nrhs=4,
    workload="uneven batch: 8^4, 12^3x24, 16^3x32, 2-level MG each (blocks 4^4 -> 2^4, 3^3x6, 4^3x8), "
             "eps 0.25, m0 -0.2, csw 1.0, Nvec 24, 3 + 2 sweeps, 4 Gaussian rhs per lattice, FGMRES(20) to 1e-10",
)


def measure_uneven_batch(env, args, reps=5):
    """Lattices of uneven sizes, 4 rhs each, solved (a) as one graph launch over all
    lattices (wcmg_solve_batch), (b) one graph per lattice in turn, (c) host-driven in
    turn, and (d) by plain FP64 GPU multigrid in turn; setups excluded."""
    torch, wcmg, stream, flush = env.torch, env.wcmg, env.stream, env.flush
    from paper_1904_08678_gb300 import inputs
    ub = UNEVEN_BATCH
    nr = ub["nrhs"]
    sets = {"f32_graph": [], "f32_host": [], "f64_host": []}
    bs, xs = [], []
    for k, dims in enumerate(ub["lattices"]):
        cfg = dict(WORKLOADS["c2"], dims=dims, nrhs=nr, gauge_seed=1040 + k, ortho=args.ortho)
        U, _ = make_inputs(cfg)
        b = inputs.source(dims, k, nrhs=nr)
        Ud = env.to_dev(U)
        bs.append(env.to_dev(b))
        xs.append(torch.zeros_like(bs[-1]))
        for name, inner, g in (("f32_graph", "f32", 1), ("f32_host", "f32", 0), ("f64_host", "f64", 0)):
            c = wcmg.Context(params(wcmg, cfg, inner, profile=0, graphs=g))
            c.set_gauge(Ud, stream)
            c.setup_seeded(cfg["gauge_seed"], stream)
            sets[name].append(c)

    def timed(fn):
        for _ in range(2):
            fn()
        ms, out = [], None
        for i in range(reps):
            out, t = timed_call(torch, stream, flush, fn, i)
            ms.append(t)
        return statistics.median(ms), out

    def in_turn(name):
        return lambda: [c.solve(bs[k], xs[k], nrhs=nr, stream=stream) for k, c in enumerate(sets[name])]

    res = {}
    ms, sts = timed(lambda: wcmg.Context.solve_batch(sets["f32_graph"], bs, xs, nrhs=[nr] * len(bs), stream=stream))
    res["one_graph_launch"] = {"ms": round(ms, 3), "graph": [s.graph for s in sts],
                               "outer_iterations": [s.outer_iterations for s in sts],
                               "true_residual": max(s.true_residual for s in sts),
                               "gpu_launches": sum(s.kernel_launches for s in sts)}
    for label, name in (("graph_per_lattice", "f32_graph"), ("host_driven", "f32_host"), ("fp64_host_driven", "f64_host")):
        ms, sts = timed(in_turn(name))
        res[label] = {"ms": round(ms, 3), "outer_iterations": [s.outer_iterations for s in sts],
                      "true_residual": max(s.true_residual for s in sts)}
    for v in sets.values():
        for c in v:
            c.close()
    res["workload"] = ub["workload"]
    res["speedup_vs_fp64"] = round(res["fp64_host_driven"]["ms"] / res["one_graph_launch"]["ms"], 2)
    res["reps"] = reps
    return res


# ---------------------------------------------------------------- oracle
# The FP64 numpy oracle cannot run the 32^3x64 setup + solve inside a bench (one fine
# D application alone takes ~20 s, the whole step hours).  Its time for one step is
# therefore modelled: each oracle operator is timed on this host, and the times are
# multiplied by the number of times one step applies that operator (the GPU step's
# own operator counters).  Level-0 operators act site by site, so they are timed on a
# slab of the fine lattice (32^3 x 4: same x, y, z extents and blocks, 1/16 of the
# volume) and scaled by the volume ratio; the coarse levels are timed at full size.

ORACLE_SLAB_T = 4


def oracle_ops(cfg):
    """Callables, each one application of an oracle operator of the workload (built on
    the slab for level 0, at full size for the coarse levels), with the factor that
    scales one call to the full lattice."""
    from oracle.aggregation import Aggregation
    from oracle.coarse import CoarseOperator
    from oracle.lattice import coarse_dims, to_grid
    from oracle.wilson import WilsonClover
    from paper_1904_08678_gb300 import inputs
    dims = tuple(cfg["dims"])
    slab = dims[:3] + (ORACLE_SLAB_T,)
    scale0 = dims[3] / ORACLE_SLAB_T
    Vs = int(np.prod(slab))
    U = inputs.random_gauge(slab, cfg["eps"], cfg["gauge_seed"], workers=min(16, os.cpu_count() or 1))
    D = WilsonClover(U, slab, cfg["m0"], cfg["csw"])
    psi = to_grid(inputs.source(slab, cfg["source_seed"])[0].reshape(Vs, 12), slab)
    vecs0 = [to_grid(v, slab) for v in inputs.setup_vectors(slab, 12, cfg["nvec"][0], 0, cfg["gauge_seed"])]
    agg0 = Aggregation(slab, cfg["blocks"][0], vecs0)
    phi0 = agg0.restrict(psi)
    ops = {"clover_build": (lambda: WilsonClover(U, slab, cfg["m0"], cfg["csw"]), scale0),
           "apply_l0": (lambda: D(psi), scale0),
           "restrict_l0": (lambda: agg0.restrict(psi), scale0),
           "prolong_l0": (lambda: agg0.prolong(phi0), scale0),
           "ortho_l0": (lambda: Aggregation(slab, cfg["blocks"][0], vecs0), scale0)}
    ld = level_dims(cfg)
    for l in range(1, len(cfg["blocks"]) + 1):
        cd, nb = ld[l], 2 * cfg["nvec"][l - 1]
        Vc = int(np.prod(cd))
        A = inputs.complex_gaussian(900 + l, 0, (9,) + tuple(cd[::-1]) + (nb, nb))
        op = CoarseOperator(A, cd)
        phi = to_grid(inputs.complex_gaussian(901 + l, 0, (Vc, nb)), cd)
        ops[f"apply_l{l}"] = (lambda op=op, phi=phi: op(phi), 1.0)
        if l < len(cfg["blocks"]):
            vl = [to_grid(v, cd) for v in inputs.setup_vectors(cd, nb, cfg["nvec"][l], l, cfg["gauge_seed"])]
            agg = Aggregation(cd, cfg["blocks"][l], vl)
            ph = agg.restrict(phi)
            ops[f"restrict_l{l}"] = (lambda agg=agg, phi=phi: agg.restrict(phi), 1.0)
            ops[f"prolong_l{l}"] = (lambda agg=agg, ph=ph: agg.prolong(ph), 1.0)
            ops[f"ortho_l{l}"] = (lambda cd=cd, l=l, vl=vl: Aggregation(cd, cfg["blocks"][l], vl), 1.0)
    return ops


def time_op(fn):
    c0, t0 = time.process_time(), time.perf_counter()
    fn()
    return time.perf_counter() - t0, time.process_time() - c0


def model_time(times, counts, cfg):
    """Oracle seconds of one step: sum over operators of (time per call at full size) x
    (calls per step); a coarsening of level l is modelled from the oracle's own
    construction, column by column: 2 Nvec_l columns, each one application of the nine
    pieces of D_l plus nine restrictions."""
    total, parts = times["clover_build"], {"clover_build": times["clover_build"]}
    for l in range(len(cfg["blocks"]) + 1):
        for kind in ("apply", "restrict", "prolong", "ortho"):
            key = f"{kind}_l{l}"
            if key in times and counts[kind][l]:
                parts[key] = counts[kind][l] * times[key]
                total += parts[key]
        if l < len(cfg["blocks"]) and counts["coarsen"][l]:
            cols = 2 * cfg["nvec"][l]
            parts[f"coarsen_l{l}"] = counts["coarsen"][l] * cols * (times[f"apply_l{l}"] + 9 * times[f"restrict_l{l}"])
            total += parts[f"coarsen_l{l}"]
    return total, parts


def oracle_model(counts, cfg):
    """cpu_baseline of the GPU line: one timing of every oracle operator, times the
    GPU step's operator counts."""
    ops = oracle_ops(cfg)
    times, wall, cpu = {}, 0.0, 0.0
    for name, (fn, scale) in ops.items():
        w, c = time_op(fn)
        times[name] = w * scale
        wall += w
        cpu += c
    total, parts = model_time(times, counts, cfg)
    return {"value": round(total, 1), "unit": "s", "cores": max(1, round(cpu / wall)), "kind": "oracle",
            "modelled": True,
            "sample": f"each oracle operator timed once on this host ({wall:.1f} s wall): level-0 operators on a "
                      f"{cfg['dims'][0]}^3x{ORACLE_SLAB_T} slab of the fine lattice scaled by the volume ratio, "
                      "coarse levels at full size; value = sum of (time per call) x (calls in one GPU step, from the "
                      "library's operator counters); BLAS-1 and Krylov bookkeeping not counted",
            "seconds_per_call": {k: round(v, 3) for k, v in times.items()}, "seconds_per_step": {
                k: round(v, 1) for k, v in parts.items()}, "op_counts": counts, "host_cores_available": os.cpu_count()}


ONE_THREAD_ENV = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1",
                  "BLIS_NUM_THREADS": "1", "NUMEXPR_NUM_THREADS": "1", "VECLIB_MAXIMUM_THREADS": "1"}


def oracle_model_one_core(counts, workload):
    """The same operator model timed on one host core: a child process (started by exec,
    never a fork of this CUDA process) whose BLAS / OpenMP thread counts are 1 in its
    environment, pinned to one CPU where the host allows it."""
    with tempfile.NamedTemporaryFile("w", suffix=".json", delete=False) as f:
        json.dump({"counts": counts, "workload": workload}, f)
        path = f.name
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-one-core", path]
    try:
        r = subprocess.run(cmd, env=dict(os.environ, **ONE_THREAD_ENV), capture_output=True, text=True, timeout=900)
        out = json.loads(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 and r.stdout.strip() else None
    except (subprocess.TimeoutExpired, ValueError, IndexError):
        out = None
    finally:
        os.unlink(path)
    return out


def oracle_one_core_child(path):
    with open(path) as f:
        job = json.load(f)
    if hasattr(os, "sched_setaffinity"):
        try:
            os.sched_setaffinity(0, {min(os.sched_getaffinity(0))})
        except OSError:
            pass
    counts = {k: v for k, v in job["counts"].items()}
    out = oracle_model(counts, dict(WORKLOADS[job["workload"]]))
    print(json.dumps({"value": out["value"], "unit": "s", "cores": 1, "cores_measured": out["cores"],
                      "seconds_per_call": out["seconds_per_call"]}), flush=True)


def run_reference(args, rank, world):
    """The oracle arm: its modelled time-to-solution for the workload's step.  Each of the
    W + K steps times one oracle operator (round robin); value = the model from the
    timed steps' samples (an operator sampled only in warm-up uses that sample)."""
    if world > 1:
        dist = dist_init(world, "gloo")
        if rank != 0:
            barrier(dist)
            dist.destroy_process_group()
            return
    else:
        dist = None
    cfg = dict(WORKLOADS[args.workload])
    counts = OP_COUNTS.get(args.workload)
    if counts is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no recorded operator counts for workload "
                                                              f"{args.workload}"}), flush=True)
        return
    ops = oracle_ops(cfg)
    names = list(ops)
    timed, warm = {k: [] for k in names}, {k: [] for k in names}
    wall, cpu = 0.0, 0.0
    for i in range(args.warmup + args.steps):
        name = names[i % len(names)]
        fn, scale = ops[name]
        w, c = time_op(fn)
        (timed if i >= args.warmup else warm)[name].append(w * scale)
        wall += w
        cpu += c
    times = {k: statistics.median(timed[k] or warm[k]) for k in names if timed[k] or warm[k]}
    missing = [k for k in names if k not in times]
    for k in missing:  # fewer steps than operators: time the rest once now
        w, c = time_op(ops[k][0])
        times[k] = w * ops[k][1]
    total, parts = model_time(times, counts, cfg)
    v = round(total, 1)
    line = {"impl": "reference", "metric": "time_to_solution_1e-10", "value": v, "unit": "s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["workload"], "dims": list(cfg["dims"]), "inner_prec": "f64"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": max(1, round(cpu / max(wall, 1e-9))), "kind": "oracle",
                             "modelled": True,
                             "sample": f"each step times one oracle operator (round robin over {len(names)}): "
                                       f"level-0 operators on a {cfg['dims'][0]}^3x{ORACLE_SLAB_T} slab scaled by "
                                       "the volume ratio, coarse levels at full size; value = sum of (median time "
                                       "per call) x (calls per step recorded by the GPU arm's operator counters)"},
            "seconds_per_call": {k: round(x, 3) for k, x in times.items()},
            "seconds_per_step": {k: round(x, 1) for k, x in parts.items()},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if dist is not None:
        barrier(dist)
        dist.destroy_process_group()


def run_table2(args, rank, world, local):
    """Setup-vs-solve trade-off of Table 2 on the synthetic 16^4 field: for 0..10
    refinement sweeps, the initial-setup, iterative-setup and solve times and the outer
    iterations (the paper's columns), each the median of 3 steps after 2 warm-up steps."""
    import torch
    from paper_1904_08678_gb300 import wcmg
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush = L2Flush(torch, dev)
    cfg = dict(WORKLOADS["table2"])
    U, b = make_inputs(cfg)
    Ud, bd = (torch.from_numpy(a).to(dev) for a in (U, b))
    xd = torch.zeros_like(bd)
    rows = []
    with ClockSampler(local) as clk:
        for sweeps in range(11):
            c = dict(cfg, refine_sweeps=sweeps)
            ctx = wcmg.Context(params(wcmg, c, args.inner, args.links, graphs=args.graphs))
            res = []
            for i in range(5):
                flush.fill_(i)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.set_gauge(Ud, stream)
                s1 = ctx.setup_seeded(cfg["gauge_seed"], stream)
                s2 = ctx.solve(bd, xd, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                res.append((e0.elapsed_time(e1), s1, s2))
            res = res[2:]
            med = lambda f: round(statistics.median(f(r) for r in res), 2)
            rows.append({"setup_iter": sweeps, "outer_iterations": res[-1][2].outer_iterations,
                         "initial_setup_ms": med(lambda r: r[1].ms_setup_init),
                         "iterative_setup_ms": med(lambda r: r[1].ms_setup_refine),
                         "solve_ms": med(lambda r: r[2].ms_solve), "total_ms": med(lambda r: r[0]),
                         "true_residual": max(r[2].true_residual for r in res)})
            ctx.close()
    best = min(rows, key=lambda r: r["total_ms"])
    line = {"metric": "time_to_solution_1e-10", "value": round(best["total_ms"] / 1e3, 5), "unit": "s",
            "n_gpus": 1, "steps": 3, "warmup": 2, "ms_per_step": best["total_ms"], "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.inner == "f32" else "f64",
            "data": "synthetic", "config": {"workload": cfg["workload"], "best_setup_iter": best["setup_iter"],
                                            "inner_prec": args.inner},
            "table2": rows, "clocks": clk.summary(), "roofline": None,
            "note": "a parameter sweep; per-kernel rooflines are in the 16^3x32 line"}
    print(json.dumps(line), flush=True)


def run_probe(args, local):
    """One kernel family of the workload, isolated, for an ncu capture on a small case:
    'ortho' runs wcmg_set_nullvecs on the fine level (its FP64 or double-float block
    orthonormalisation) 3 times; 'coarse:L:N' runs one setup, then 5 coarse applies of level
    L with N rhs (the autotuned launch shape)."""
    import torch
    torch.cuda.set_device(local)
    env = Env(local, None)
    torch_, wcmg, stream = env.torch, env.wcmg, env.stream
    cfg = dict(WORKLOADS[args.workload])
    if args.links:
        cfg["links"] = args.links
    cfg["ortho"] = args.ortho
    if args.sigma3:
        cfg["sigma3"] = 1
    if args.probe_fine:
        # a smaller fine lattice whose first blocking gives the same coarse levels (the
        # coarse applies' shapes and bytes unchanged, the device memory much smaller)
        d, b = args.probe_fine.split("/")
        cfg["dims"] = tuple(int(x) for x in d.split("x"))
        cfg["blocks"] = [tuple(int(x) for x in b.split("x"))] + list(cfg["blocks"][1:])
        cfg["workload"] += f"; fine lattice replaced by {d} with blocks {b} for the probe"
    from paper_1904_08678_gb300 import inputs
    ld = level_dims(cfg)
    out = {"probe": args.probe, "workload": cfg["workload"], "ortho": args.ortho}
    if args.probe == "clover":
        ctx = wcmg.Context(params(wcmg, cfg, "f32", profile=1 << KCLASS.index("clover"), nrhs=1))
        U, _ = make_inputs(cfg, 1)
        ctx.set_gauge(env.to_dev(U), stream)
        k0 = ctx.kstats()["clover"]
        ms = [timed_call(torch_, stream, env.flush, lambda: ctx.set_clover(cfg["csw"], stream), i)[1]
              for i in range(3)]
        k1 = ctx.kstats()["clover"]
        out.update(ms_per_call=[round(t, 3) for t in ms],
                   kernel_ms=round((k1["ms"] - k0["ms"]) / max(k1["launches"] - k0["launches"], 1), 3))
    elif args.probe.startswith("dslash"):
        # the FP32 fine stencil alone: wcmg_apply_D with N rhs (its packing kernels are
        # another class), 5 calls with L2 flushed before each
        nr = int(args.probe.split(":")[1]) if ":" in args.probe else 1
        ctx = wcmg.Context(params(wcmg, cfg, "f32", profile=1 << KCLASS.index("dslash"), nrhs=nr))
        U, _ = make_inputs(cfg, 1)
        ctx.set_gauge(env.to_dev(U), stream)
        V = int(np.prod(ld[0]))
        x = env.to_dev(inputs.complex_gaussian(33, 0, (nr, V, 12)))
        y = torch_.zeros_like(x)
        ctx.apply_D(x, y, nrhs=nr, prec=wcmg.F32, stream=stream)
        k0 = ctx.kstats()["dslash"]
        if args.ncu_region:
            torch_.cuda.profiler.start()
        ms = [timed_call(torch_, stream, env.flush,
                         lambda: ctx.apply_D(x, y, nrhs=nr, prec=wcmg.F32, stream=stream), i)[1] for i in range(5)]
        if args.ncu_region:
            torch_.cuda.profiler.stop()
        k1 = ctx.kstats()["dslash"]
        kus = (k1["ms"] - k0["ms"]) / max(k1["launches"] - k0["launches"], 1) * 1e3
        algo = V * (nr * 192 + 576)
        out.update(nrhs=nr, ms_per_call=[round(t, 3) for t in ms], kernel_us=round(kus, 2), algorithmic_bytes=algo,
                   frac_of_hbm=round(algo / (kus * 1e-6) / 1e9 / peaks()[0], 4))
    elif args.probe == "ortho":
        nv = cfg["nvec"][0]
        ctx = wcmg.Context(params(wcmg, cfg, "f32", profile=1 << KCLASS.index("ortho"), nrhs=1))
        V = int(np.prod(ld[0]))
        vecs = env.to_dev(inputs.complex_gaussian(31, 0, (nv, V, 12)))
        ms = [timed_call(torch_, stream, env.flush, lambda: ctx.set_nullvecs(0, vecs, stream), i)[1] for i in range(3)]
        k = ctx.kstats()["ortho"]
        out.update(ms_per_call=[round(t, 3) for t in ms], kernel_ms=round(k["ms"] / max(k["launches"], 1), 3),
                   gflop_per_launch=round(k["flops"] / max(k["launches"], 1) / 1e9, 2))
    else:
        fields_ = args.probe.split(":")
        lev, nr = int(fields_[1]), int(fields_[2])
        forced = [int(x) for x in fields_[3:]]  # optional kind:threads:parts:stages:ntile
        U, b = make_inputs(cfg, 1)
        ctx = wcmg.Context(params(wcmg, cfg, "f32", profile=0, autotune=1, nrhs=max(nr, 1)))
        ctx.set_gauge(env.to_dev(U), stream)
        ctx.setup_seeded(cfg["gauge_seed"], stream)
        Vc, nb = int(np.prod(ld[lev])), 2 * cfg["nvec"][lev - 1]
        phi = env.to_dev(inputs.complex_gaussian(32, 0, (nr, Vc, nb)))
        y = torch_.zeros_like(phi)
        if forced:
            f = forced + [0] * (5 - len(forced))
            ctx.set_coarse_tile(lev, nr, wcmg.F32, kind=f[0], threads=f[1], parts=f[2], stages=f[3], ntile=f[4])
        ctx.apply_coarse(lev, phi, y, nrhs=nr, prec=wcmg.F32, stream=stream)  # autotune (unless forced)
        ctx.set_profile(1 << KCLASS.index("coarse"))
        k0 = ctx.kstats()["coarse"]
        if args.ncu_region:
            torch_.cuda.profiler.start()  # ncu --profile-from-start off: the timed applies only
        ms = [timed_call(torch_, stream, env.flush,
                         lambda: ctx.apply_coarse(lev, phi, y, nrhs=nr, prec=wcmg.F32, stream=stream), i)[1]
              for i in range(5)]
        if args.ncu_region:
            torch_.cuda.profiler.stop()
        k1 = ctx.kstats()["coarse"]
        n = max(k1["launches"] - k0["launches"], 1)
        kus = (k1["ms"] - k0["ms"]) / n * 1e3
        lb = {"f32": 8, "bf16": 4, "f16": 4}[cfg.get("links", "f32")]
        algo = Vc * (9 * nb * nb * lb + 2 * nb * 8 * nr)
        out.update(level=lev, nrhs=nr, tile=ctx.get_coarse_tile(lev, nr, wcmg.F32), ms_per_call=[round(t, 3) for t in ms],
                   kernel_us=round(kus, 2), algorithmic_bytes=algo,
                   frac_of_hbm=round(algo / (kus * 1e-6) / 1e9 / peaks()[0], 4))
    ctx.close()
    print(json.dumps(out), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--inner", default="f32", choices=["f32", "f64"])
    ap.add_argument("--links", default=None, choices=["f32", "bf16", "f16"],
                    help="coarse-link storage (default: the workload's own)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-one-core", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-sub", action="store_true", help="headline workload only, no sub-records")
    ap.add_argument("--sub-steps", type=int, default=3, help="timed steps of each sub-record")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--nrhs", type=int, default=0, help="override the workload's number of right-hand sides")
    ap.add_argument("--graphs", type=int, default=1, choices=[0, 1],
                    help="1: each solve replays one captured CUDA graph; 0: host-driven solve")
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                    help="1: coarse-apply launch shapes picked by the autotuner; 0: fixed rule")
    ap.add_argument("--kcycle", action="store_true", help="K-cycle on the intermediate levels (3-level workloads)")
    ap.add_argument("--coarse-eo", action="store_true",
                    help="even-odd (Schur complement) preconditioned coarsest solve")
    ap.add_argument("--sigma3", action="store_true",
                    help="keep five-block (sigma3) copies of the Galerkin coarse links: the autotuner may pick the "
                         "five-block one-rhs apply (kind 5); coarse_stencil reports it with its own byte count")
    ap.add_argument("--smoother", default="mr", choices=["mr", "gmres", "sap"],
                    help="smoother of every level (the setup sweeps and the cycle)")
    ap.add_argument("--sap-cycles", type=int, default=1, help="SAP smoother: cycles")
    ap.add_argument("--smoother-steps", type=int, default=4, help="MR / GMRES steps (SAP: MR steps per block)")
    ap.add_argument("--sap-eo", action="store_true", help="SAP: even-odd preconditioned block solves (fine level)")
    ap.add_argument("--pools", type=int, default=417,
                    help="c5: training pools of 48 fresh pairs (417 pools = 20016 pairs)")
    ap.add_argument("--ortho", default="df", choices=["fp64", "df"],
                    help="block orthonormalisation arithmetic of the FP32-inner runs: double-float on the FP32 "
                         "pipe (default; the same Q to 1e-14) or FP64; plain FP64 multigrid always uses FP64")
    ap.add_argument("--probe", default=None,
                    help="kernel probe for ncu instead of the bench: 'clover' (the clover term of the "
                         "workload's gauge field, 3 times), 'ortho' (the fine-level block "
                         "orthonormalisation of Nvec Gaussian fields, 3 times), 'dslash:NRHS' (the FP32 fine stencil "
                         "through wcmg_apply_D, 5 calls) or 'coarse:LEVEL:NRHS[:KIND:THREADS:"
                         "PARTS:STAGES:NTILE]' (5 coarse applies after one setup with the autotuned or the given "
                         "launch shape); prints one JSON line of CUDA-event times")
    ap.add_argument("--probe-fine", default=None,
                    help="probe only: replace the fine lattice and its blocking, e.g. 12x12x12x24/2x2x2x2 keeps "
                         "the 24^3x48 workload's 6^3x12 level 1 on a fine lattice 8x smaller")
    ap.add_argument("--ncu-region", action="store_true",
                    help="bracket the timed steps of the headline workload (or a coarse probe's timed applies) "
                         "with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    args = ap.parse_args(argv)
    if args.oracle_one_core:  # the child of oracle_model_one_core (CPU only)
        oracle_one_core_child(args.oracle_one_core)
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    rank, world, local = dist_env()
    if args.probe:
        run_probe(args, local)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "table2":
        run_table2(args, rank, world, local)
    else:
        run_gpu(args, rank, world, local)


if __name__ == "__main__":
    main()
