"""Benchmark: voxel-iterations/s of the ComBo FFT homogenization hot path on GB300.

Workload (default): 256^3 periodic grid of seeded random non-overlapping
balls of radius 12 voxels at volume fraction 0.25, Neo-Hookean contrast 100,
uniaxial stretch to Fbar11 = 1.10 in 10 load steps; Newton-CG with FP32
Krylov iterations, FP64 laminate solves, FP64 constitutive law and norms,
residual transforms in double-float arithmetic (``--precision refined``
keeps them in FP64, ``--precision fp64`` runs every operator in FP64).

A step is one operator application of the solve -- one voxel-iteration per
voxel: tangent (or constitutive law + boxel laminates), forward FFT, Green
operator, inverse FFT, Krylov update -- with the amortised FP64 residual
evaluations and laminate solves the solver interleaves.  ``value`` counts
the operator applications the solve actually ran inside the timed region,
which starts at a Newton step boundary and runs on to the end of the Newton
step in which K operator applications are reached, so the residual
evaluation and laminate solves of every Newton step it touches are inside.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl combo|reference]

N > 1 runs N independent replicas, one per GPU (the path does not shard; no
data-path collective), under torchrun; rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel-iterations/s"
WORKLOAD = "spheres_256"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=24)
    ap.add_argument("--impl", default="combo", choices=["combo", "reference"])
    ap.add_argument("--precision", default="refined-df", choices=["refined-df", "refined", "fp64"])
    ap.add_argument("--n", type=int, default=256, help="grid side (256 = the benchmark workload)")
    ap.add_argument("--shape", default=None, help="n1,n2,n3 of a smaller ball grid (profiling captures)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the plain FP64 solve that states the refined form's accuracy")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-fibres", action="store_true", help="skip the 512^3 fibre workload")
    ap.add_argument("--no-normals", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--normals-only", default=None, metavar="N1,N2,N3",
                    help="only coarse-grain a seeded spheres image of this size (8^3 boxels), three calls "
                         "(profiling captures of the coarse-graining kernels)")
    ap.add_argument("--serve-full", action="store_true",
                    help="120 requests (24 of them in all three precision forms; takes many minutes)")
    ap.add_argument("--serve-only", action="store_true", help="only the serving section")
    ap.add_argument("--profile-json", default=None, help="write the per-kernel table here")
    ap.add_argument("--batch-only", action="store_true", help="only the 64-solve batch section")
    ap.add_argument("--fibres-only", action="store_true", help="only the 512^3 fibre section")
    ap.add_argument("--variants-only", action="store_true", help="only the solver / discretisation variants")
    ap.add_argument("--dfmg-only", type=int, default=0, metavar="N",
                    help="only the doubly-fine material grid kernel timings on an N^3 random-ball problem")
    ap.add_argument("--krylov-form", default="nodal", choices=["nine", "displacement", "nodal"],
                    help="most reduced evaluation form of the rotated Krylov operator")
    return ap.parse_args()


def workload(n, shape=None):
    from paper_2204_13624_gb300 import microstructure as ms

    if shape:
        dims = tuple(int(v) for v in shape.split(","))
        return ms.random_spheres(dims, 12.0 * max(dims) / 256.0, 0.2, ms.SEED_BASE + 1, 100.0,
                                 np.diag([1.10, 1.0, 1.0]), 10)
    if n == 256:
        return ms.spheres_256()
    return ms.spheres_256(n=n, vf=0.2 if n >= 128 else 0.1)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, nm in enumerate(names):
                if len(s) > 5 + k and s[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ---------------------------------------------------------------- roofline
def algorithmic_bytes(kernel, p, krylov_bytes, disp=False, nodal=False):
    """Bytes the method must move per launch of a kernel class (reads + writes
    of the fields it touches, each once), for the roofline.  disp: the Krylov
    operator runs in the displacement form (one nodal spectrum per tensor row
    leaves the z-pass; the y-inverse and x-inverse take three components; the
    gradient pass reads the three nodal fields and r, and writes r).  nodal:
    also the forward side takes three components (the tangent pass writes
    the nodal forces' spectra; the halo lines it re-reads are not counted)."""
    n1, n2, n3 = p["n"]
    V = n1 * n2 * n3
    nb = int(p["boxel_idx"].size)
    nh = n1 // 2 + 1
    spec_c = 9 * n3 * n2 * nh  # stored half-spectrum complex entries
    w = krylov_bytes
    if kernel == "xfwd_nodal":
        return V * (45 * w + 1) + (V - nb) * 10 * w + nb * (4 + 45 * w) + (spec_c // 3) * 2 * w
    if nodal and kernel in ("yfwd_krylov", "zgamma_krylov"):
        return 2 * (spec_c // 3) * 2 * w
    if disp and kernel == "zgamma_krylov":
        return (spec_c + spec_c // 3) * 2 * w
    if disp and kernel == "yinv_krylov":
        return 2 * (spec_c // 3) * 2 * w
    if disp and kernel == "xinv_cg":
        # three spectra read, three real nodal fields written
        return (spec_c // 3) * 2 * w + 3 * V * w
    if kernel == "grad_cg":
        # nodal fields read, r read + written
        return 3 * V * w + V * 18 * w
    if kernel == "xinv_grad_cg":
        # three spectra read; r read + written (the nodal fields stay on chip)
        return (spec_c // 3) * 2 * w + V * 18 * w
    if kernel in ("yfwd_krylov", "zgamma_krylov", "yinv_krylov"):
        return 2 * spec_c * 2 * w
    if kernel in ("yfwd_fp64", "zgamma_fp64", "yinv_fp64"):
        return 2 * spec_c * 16
    if kernel == "xfwd_tangent":
        # r, p, x read; p, x written (x += alpha p of the previous iteration);
        # tangent cache (9 + 1 words) at pure voxels; phase byte; boxel voxel
        # index and packed symmetric 45-entry tangent at boxels; spectrum written
        return V * (45 * w + 1) + (V - nb) * 10 * w + nb * (4 + 45 * w) + spec_c * 2 * w
    if kernel == "xinv_cg":
        # spectrum read; r read + written
        return spec_c * 2 * w + V * 18 * w
    if kernel == "xfwd_resid_fp64":
        # F read (FP64), phase, P_box at boxels, tangent cache written, spectrum written
        return V * (72 + 1) + nb * (4 + 72) + (V - nb) * 10 * w + spec_c * 16
    if kernel == "xinv_fp64":
        return spec_c * 16 + V * 18 * w
    if kernel == "boxel_laminate":
        return nb * (4 + 72 + 24 + 8 + 24 * 2 + 72 + 4 + 45 * w)
    return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(kernel, alg_bytes):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (profiles/ncu_traffic_<kernel>_*.txt): the captured traffic / algorithmic
    ratio times this workload's algorithmic bytes, or None when the kernel's
    sources changed after the capture."""
    import glob
    import hashlib

    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", f"ncu_traffic_{kernel}_*.txt"))):
        kv = {}
        for line in open(path):
            if line.startswith("#") or ":" not in line:
                continue
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
        if kv.get("kernel") != kernel or not alg_bytes:
            continue
        h = hashlib.sha256()
        d = os.path.join(ROOT, "paper_2204_13624_gb300", "csrc")
        try:
            for f in kv["sources"].split():
                h.update(open(os.path.join(d, f), "rb").read())
        except OSError:
            return None
        if h.hexdigest()[:16] != kv.get("sources_sha256_16"):
            return None
        return float(kv["traffic_over_algorithmic"]) * alg_bytes
    return None


# ---------------------------------------------------------------- replicas
def replicas_aggregate(ms, ops, dist, device):
    """Whole-job figures of N independent replicas (one per rank, no data-path
    collective): the longest timed region over the ranks and the operator
    applications of all ranks.  dist None: the rank's own figures."""
    if dist is None:
        return ms, ops
    import torch

    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    o = torch.tensor([float(ops)], device=device, dtype=torch.float64)
    dist.all_reduce(o, op=dist.ReduceOp.SUM)
    return float(t.item()), int(o.item())


# ---------------------------------------------------------------- CPU baseline
def oracle_cg_rate(p, base, extra, cores, reps=1):
    """Oracle (FP64, OpenMP over the host cores) CG operator applications of
    its Newton-CG on the first load step -- the operation `value` counts on
    the GPU: tangent, FFT, Green operator, inverse FFT, CG update -- timed as
    the difference of a run with base + extra and one with base CG iterations
    in its one Newton step, so set-up, residual and laminate solves cancel.
    With reps > 1 the two runs alternate reps times and the fastest of each
    enters the difference; a difference that host noise still leaves at or
    below zero is measured again with four times the extra iterations (up to
    twice)."""
    import oracle

    def run(iters):
        t0 = time.perf_counter()
        r = oracle.solve(dict(p, n_steps=1), dict(solver=1, fixed_iter=1, cg_fixed_iter=iters, nthreads=cores),
                         fields=False)
        return time.perf_counter() - t0, int(r["n_operator"])

    V = p["n"][0] * p["n"][1] * p["n"][2]
    for _ in range(3):
        t_base, t_more = [], []
        for _ in range(max(reps, 1)):
            tb, n0 = run(base)
            tm, n1 = run(base + extra)
            t_base.append(tb)
            t_more.append(tm)
        dt = min(t_more) - min(t_base)
        ops = n1 - n0
        if dt > 0:
            break
        extra *= 4
    return ops, dt, (ops * V / dt if dt > 0 else None)


def cpu_baseline(p, iters=1):
    """The oracle as it stands on the same workload for a bounded number of CG
    operator applications (oracle_cg_rate)."""
    cores = len(os.sched_getaffinity(0))
    ops, dt, value = oracle_cg_rate(p, 1, iters, cores)
    return {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{ops} CG operator application(s) of the oracle's Newton-CG on the {WORKLOAD} workload, "
                      f"first load step, FP64: the difference of runs with {1 + iters} and 1 CG iterations "
                      f"(set-up, residual and laminate solves cancelled)",
            "seconds": dt}


# ---------------------------------------------------------------- main
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2204_13624_gb300 import build as cbuild
    from paper_2204_13624_gb300 import combo

    if rank == 0 or world == 1:
        cbuild.build()
    if dist:
        dist.barrier()
    combo.load()
    combo.krylov_form({"nine": 0, "displacement": 1, "nodal": 2}[args.krylov_form])
    # one explicit stream for torch and the library, so that the CUDA events
    # bracket the library's launches and torch's allocations are ordered
    # with them (the default stream's handle would give the library its own)
    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    ctx = combo.Context(local, stream.cuda_stream)
    if args.dfmg_only:
        from paper_2204_13624_gb300 import microstructure as ms

        n = args.dfmg_only
        p = ms.random_spheres((n, n, n), 8.0, 0.2, ms.SEED_BASE + 6, 10.0, np.diag([1.05, 1.0, 1.0]), 2)
        print(json.dumps({"dfmg_only": n, "dfmg_kernels": dfmg_kernels(combo, ctx, p)}))
        return
    if args.serve_only:
        print(json.dumps({"serving": serving_bench(combo, ctx, count=120, compare=24) if args.serve_full
                          else serving_bench(combo, ctx)}))
        return
    if args.fibres_only:
        peak, peak_kind = peaks()
        print(json.dumps({"fibres_512": fibres_bench(combo, ctx, stream, peak, peak_kind)}))
        return
    if args.variants_only:
        print(json.dumps({"variants": variants_bench(combo, ctx)}))
        return
    if args.batch_only:
        print(json.dumps({"batch": batch_bench(combo, ctx)}))
        return
    if args.normals_only:
        from paper_2204_13624_gb300 import microstructure as ms

        n = tuple(int(v) for v in args.normals_only.split(","))
        d = torch.from_numpy(ms.fine_spheres_image(n, 24, max(1, int(4000 * np.prod(n) / 1024**3)),
                                                   seed=ms.SEED_BASE + 5)).cuda()
        for _ in range(3):
            nb = combo.coarse_grain(d, (8, 8, 8), ctx=ctx)[4]
        torch.cuda.synchronize()
        print(json.dumps({"normals_only": list(n), "boxels": int(nb)}))
        return
    p = workload(args.n, args.shape)
    V = p["n"][0] * p["n"][1] * p["n"][2]
    prec = {"refined": combo.FP32_REFINED, "refined-df": combo.FP32_REFINED_DF, "fp64": combo.FP64}[args.precision]
    clk = ClockSampler(local)
    ms, ops, residuals, prof, done = timed_window(combo, ctx, p, prec, args.steps, args.warmup, stream, dist, clk)
    clocks = clk.stop()
    t_max, ops_all = replicas_aggregate(ms, ops, dist, "cuda")
    value = ops_all * V / (t_max / 1e3)
    peak, peak_kind = peaks()
    table, roof, cg_ms, newton_ms, launches = kernel_table(combo, prof, p, prec, ops, peak, peak_kind)

    e2e = None
    if not args.no_e2e and rank == 0:
        e2e = run_e2e(p, prec, combo, ctx, V)
        if prec != combo.FP64 and world == 1 and not args.no_fp64_compare:
            # the plain FP64 form of the same solve: the stated accuracy of
            # this form against it, and the speed-up at equal tolerance
            ref = run_e2e(p, combo.FP64, combo, ctx, V)
            a, b = np.asarray(e2e.pop("_Pbar")), np.asarray(ref.pop("_Pbar"))
            e2e["Pbar_rel_err_vs_fp64"] = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
            e2e["Pbar_rel_err_vs_fp64_final_step"] = float(np.max(np.abs(a[-1] - b[-1])) / np.max(np.abs(b[-1])))
            e2e["speedup_vs_fp64"] = ref["solve_seconds"] / e2e["solve_seconds"]
            e2e["fp64"] = ref
        e2e.pop("_Pbar", None)
    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        cpu = cpu_baseline(p)
    serving = None
    if not args.no_serving and rank == 0:
        if args.serve_full:
            serving = serving_bench(combo, ctx, count=120, compare=24)
        else:
            serving = serving_bench(combo, ctx)
    batch = None
    if not args.no_batch and rank == 0:
        batch = batch_bench(combo, ctx)
    fibres = None
    if not args.no_fibres and rank == 0:
        fibres = fibres_bench(combo, ctx, stream, peak, peak_kind)
    variants = None
    if not args.no_variants and rank == 0:
        variants = variants_bench(combo, ctx)
    normals = None
    if not args.no_normals and rank == 0:
        normals = normals_bench(combo, ctx, stream, peak, peak_kind, cpu=not args.no_cpu_baseline and world == 1)

    arith = None
    if rank == 0:
        # FP64 / FP32 FMA rates of this GPU: the ceilings of the kernels bound by arithmetic
        r64, r32 = combo.arith_rates(ctx)
        arith = {"fp64_tflops": r64, "fp32_tflops": r32, "fp32_over_fp64": (r32 / r64) if r64 > 0 else None,
                 "method": "combo_arith_rates: 8 dependent FMA chains per thread, 2048 threads per SM, "
                           "CUDA events, best of 3"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / max(ops, 1),
                "ms_per_cg_iteration": cg_ms / max(ops, 1),
                "newton_residual_ms_per_step": newton_ms / max(residuals, 1), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if prec == combo.FP64 else "f32",
                "data": "synthetic",
                "config": {"workload": (f"spheres_{args.shape.replace(',', 'x')}" if args.shape else
                                        (WORKLOAD if args.n == 256 else f"spheres_{args.n}")),
                           "grid": list(p["n"]), "voxels": V, "boxels": int(p["boxel_idx"].size),
                           "microstructure": "seeded RSA balls r=12 vox, vf 0.25, contrast 100",
                           "load": "Fbar11 = 1.10 in 10 steps",
                           "solver": "Newton-CG, tol 1e-8, cg_tol 1e-3",
                           "precision": {combo.FP32_REFINED: "FP32 Krylov + FP64 residual/laminates/norms",
                                         combo.FP32_REFINED_DF: "FP32 Krylov + double-float residual transforms, "
                                                                "FP64 P(F)/laminates/norms",
                                         combo.FP64: "FP64"}[prec],
                           "kspace": "rotated (HEX8R)",
                           "operator_applications": int(ops), "newton_residuals_in_timed_region": int(residuals),
                           "timed_region": "whole Newton steps: from a Newton step boundary on to the end of the "
                                           "Newton step in which --steps operator applications are reached",
                           "solve_finished_in_timed_region": bool(done),
                           "l2": "inputs larger than L2 (each 9-field >= 604 MB)",
                           "autotune": combo.autotune_report().strip().splitlines(),
                           "parallelism": f"replicas x{world}"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "serving": serving, "batch": batch,
                "fibres_512": fibres,
                "normal_detection": normals, "variants": variants, "gpu_launches": launches,
                "clocks": clocks, "kernels": table, "arith_rates": arith}
        if args.profile_json:
            json.dump(line, open(args.profile_json, "w"), indent=1)
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def timed_window(combo, ctx, p, prec, steps, warmup, stream, dist=None, clk=None):
    """CUDA-event time of a window of whole Newton steps of one solve: after
    warm-up Newton steps (at least `warmup` operator applications), from a
    Newton step boundary on to the end of the Newton step in which `steps`
    operator applications are reached, so the residual evaluation and
    laminate solves of every Newton step it touches are inside.  Per-kernel
    CUDA events on the solve's stream are recorded over the window."""
    import torch

    s = combo.Solve(p, ctx=ctx, solver=combo.NEWTON_CG, precision=prec, tol=1e-8)
    s.advance_newton(max(warmup, 3))
    torch.cuda.synchronize()
    r0 = s.finish(fields=False)
    ops0, res0 = r0["n_operator"], r0["n_operator_fp64"]
    s.profile(True)
    if clk:
        clk.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    done = s.advance_newton(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    res = s.finish(fields=False)
    ops = res["n_operator"] - ops0
    residuals = res["n_operator_fp64"] - res0
    prof = s.profile_read()
    s.profile(False)
    s.close()
    return ms, ops, residuals, prof, done


KRYLOV = ("xfwd_tangent", "xfwd_nodal", "yfwd_krylov", "zgamma_krylov", "yinv_krylov", "xinv_cg", "grad_cg",
          "xinv_grad_cg")


def kernel_table(combo, prof, p, prec, ops, peak, peak_kind):
    """Per-kernel table of a timed window and the dominant kernel's roofline."""
    kb = 8 if prec == combo.FP64 else 4
    table = {}
    for k, (kms, cnt) in prof.items():
        if cnt == 0:
            continue
        b = algorithmic_bytes(k, p, kb,
                              disp=prof.get("grad_cg", (0.0, 0))[1] > 0 or prof.get("xinv_grad_cg", (0.0, 0))[1] > 0,
                              nodal=prof.get("xfwd_nodal", (0.0, 0))[1] > 0)
        # CG kernels are launched in graph chunks of 8 iterations; launches
        # past the converged iteration return at once and do no work, so the
        # per-launch time divides by the iterations that ran (ops)
        work = min(cnt, ops) if k in KRYLOV else cnt
        per = kms / work if work else 0.0
        table[k] = {"ms_total": kms, "launches": cnt, "launches_with_work": work, "ms_per_launch": per,
                    "alg_bytes_per_launch": b, "GBps": (b / (per / 1e3) / 1e9) if (b and per > 0) else None}
    hot = {k: v for k, v in table.items() if v["alg_bytes_per_launch"] and k not in ("boxel_laminate",)}
    dom = max(hot, key=lambda k: hot[k]["ms_total"]) if hot else None
    launches = int(sum(v["launches"] for v in table.values()))
    cg_ms = sum(table[k]["ms_total"] for k in KRYLOV if k in table)
    newton_ms = sum(v["ms_total"] for k, v in table.items() if k not in KRYLOV)
    roof = None
    if dom:
        ach = table[dom]["GBps"]
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_kind": peak_kind,
                "traffic": ncu_traffic(dom, table[dom]["alg_bytes_per_launch"]),
                "alg_bytes_per_launch": table[dom]["alg_bytes_per_launch"]}
    return table, roof, cg_ms, newton_ms, launches


def fibres_bench(combo, ctx, stream, peak, peak_kind, steps=40, warmup=8):
    """The 512^3 fibre workload (z-fibres of radius 10 voxels, fibre fraction
    0.3, contrast 50, simple shear Fbar12 = 0.15 in 15 steps; FP32 fields with
    double-float residuals, FP64 laminates and norms): a timed window of whole
    Newton steps, its kernel table and the dominant kernel's roofline."""
    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.fibres_512()
    V = p["n"][0] * p["n"][1] * p["n"][2]
    prec = combo.FP32_REFINED_DF
    t, ops, residuals, prof, _ = timed_window(combo, ctx, p, prec, steps, warmup, stream)
    table, roof, cg_ms, newton_ms, _ = kernel_table(combo, prof, p, prec, ops, peak, peak_kind)
    return {"workload": "fibres_512", "voxels": V, "boxels": int(p["boxel_idx"].size),
            "value": ops * V / (t / 1e3), "unit": METRIC, "ms_window": t, "operator_applications": int(ops),
            "newton_residuals": int(residuals), "ms_per_cg_iteration": cg_ms / max(ops, 1),
            "newton_residual_ms_per_step": newton_ms / max(residuals, 1), "roofline": roof, "kernels": table}


def run_e2e(p, prec, combo, ctx, V):
    """The user's call: combo_solve of the full problem from host buffers
    (inputs copied in, Pbar and the F and P fields copied out), wall clock."""
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = combo.solve(p, ctx=ctx, fields=True, solver=combo.NEWTON_CG, precision=prec, tol=1e-8)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ops = int(r["n_operator"])
    nb = int(p["boxel_idx"].size)
    h2d = V + nb * (8 + 24 + 8)
    d2h = 9 * 8 * len(r["Pbar"]) + 2 * 72 * V + 24 * nb
    return {"value": ops * V / dt, "unit": METRIC, "h2d_bytes_per_step": h2d / max(ops, 1),
            "d2h_bytes_per_step": d2h / max(ops, 1), "solve_seconds": dt, "operator_applications": ops,
            "fp64_residuals": int(r["n_operator_fp64"]), "load_steps": int(r["steps_done"]),
            "newton_iterations": [int(v) for v in r["iters"]], "cg_iterations": [int(v) for v in r["cg_iters"]],
            "Pbar_final": [float(v) for v in r["Pbar"][-1]], "_Pbar": np.asarray(r["Pbar"]).tolist(),
            "note": "one full combo_solve from host buffers; per-step bytes = totals / operator applications"}


SERVE_SIDES = (64, 72, 96, 108, 128, 144, 192, 216, 256)


def serving_problems(count, seed, sides=SERVE_SIDES, max_steps=10):
    """The request stream: grid side log-uniform in [64, 256], snapped to the
    2^a 3^b sides above; half random balls of the 256^3 workload's family
    (radius 12 voxels, vf 0.25, contrast 100, uniaxial stretch Fbar11 drawn
    in [1.02, 1.10]), half straight z-fibres of the 512^3 family (radius 10
    voxels, fibre fraction 0.3, contrast 50, simple shear Fbar12 drawn in
    [0.03, 0.15]); 1..max_steps load steps."""
    from paper_2204_13624_gb300 import microstructure as ms

    rng = np.random.default_rng(seed)
    logs = np.log(np.asarray(sides, float))
    out = []
    for i in range(count):
        side = int(sides[int(np.argmin(np.abs(logs - rng.uniform(logs[0], logs[-1]))))])
        steps = int(rng.integers(1, max_steps + 1))
        sd = int(rng.integers(1 << 30))
        Fb = np.eye(3)
        if rng.random() < 0.5:
            Fb[0, 0] = float(rng.uniform(1.02, 1.10))
            p = ms.random_spheres((side,) * 3, 12.0, 0.25, sd, 100.0, Fb, steps, gap_vox=2.0)
        else:
            Fb[0, 1] = float(rng.uniform(0.03, 0.15))
            p = ms.random_fibres((side,) * 3, 10.0, 0.3, sd, 50.0, Fb, steps, gap_vox=2.0)
        out.append(p)
    return out


def _serve(combo, ctx, probs, prec, slots, rate=None, seed=0):
    """All requests through one server: submitted at once (rate None), or at
    Poisson arrivals of the given rate; wall time, results, statistics."""
    srv = combo.Server(ctx, max_slots=slots)
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    next_t = 0.0
    tk = []
    for p in probs:
        if rate:
            next_t += rng.exponential(1.0 / rate)
            wait = next_t - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        tk.append(srv.submit(p, precision=prec, tol=1e-8))
    res = [srv.wait(t) for t in tk]
    dt = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    return dt, res, st


def serving_bench(combo, ctx, count=40, compare=6, slots=4, seed=2204_13624 + 4):
    """The request stream through the serving loop in the refined double-float
    form: saturated throughput (all submitted at once), then Poisson arrivals
    at 0.7 x that rate for p50 / p99 latency.  The first `compare` requests
    also run in the refined form with FP64 residual transforms and in plain
    FP64 (saturated), for the speed-up at equal tolerance and the Pbar error
    against plain FP64."""
    probs = serving_problems(count, seed)
    V = [int(np.prod(p["n"])) for p in probs]
    out = {"requests": count, "sides": list(SERVE_SIDES), "load_steps": "1..10", "slots": slots,
           "families": "balls r=12 vox vf 0.25 contrast 100 / z-fibres r=10 vox vf 0.3 contrast 50",
           "voxels_total": int(sum(V))}
    dt, res, st = _serve(combo, ctx, probs, combo.FP32_REFINED_DF, slots)
    rate = count / dt
    vit = sum(int(r["n_operator"]) * v for r, v in zip(res, V))
    ent = {"saturated_solves_per_s": rate, "saturated_seconds": dt, "voxel_iterations_per_s": vit / dt,
           "saturated_p50_seconds": st["p50_seconds"], "saturated_p99_seconds": st["p99_seconds"]}
    lam = 0.7 * rate
    dt2, _, st2 = _serve(combo, ctx, probs, combo.FP32_REFINED_DF, slots, rate=lam, seed=seed + 1)
    ent.update(arrival_rate_per_s=lam, solves_per_s=count / dt2, p50_seconds=st2["p50_seconds"],
               p99_seconds=st2["p99_seconds"], mean_seconds=st2["mean_seconds"],
               peak_concurrent=st2["peak_running"])
    out["refined"] = ent
    sub = probs[:compare]
    cmp = {"requests": len(sub)}
    pbar = {}
    for form, prec in (("refined", combo.FP32_REFINED_DF), ("refined_fp64_residual", combo.FP32_REFINED),
                       ("fp64", combo.FP64)):
        d, r, _ = _serve(combo, ctx, sub, prec, slots)
        cmp[form] = {"saturated_solves_per_s": len(sub) / d, "saturated_seconds": d}
        pbar[form] = [x["Pbar"] for x in r]
    for form in ("refined", "refined_fp64_residual"):
        errs = [float(np.max(np.abs(a - b)) / np.max(np.abs(b))) for a, b in zip(pbar[form], pbar["fp64"])]
        cmp[f"Pbar_rel_err_{form}_vs_fp64_max"] = max(errs)
        cmp[f"speedup_{form}_vs_fp64"] = cmp["fp64"]["saturated_seconds"] / cmp[form]["saturated_seconds"]
    out["compare_first_requests"] = cmp
    return out


def batch_bench(combo, ctx, prec=None):
    """64 independent random-ball solves, sides from {32, 48, 64, 96, 128}, 5
    load steps each, three ways, wall clock around all of them (set-up
    included): one combo_solve_batch over all 64 (one grouped launch per pass
    over the work items of every grid); one combo_solve_batch per grid size
    (stacked problems of one size, sizes one after another); the solves one
    after another."""
    import torch

    from paper_2204_13624_gb300 import microstructure as ms

    prec = combo.FP32_REFINED_DF if prec is None else prec
    probs = ms.batch_mix()
    groups = {}
    for i, p in enumerate(probs):
        groups.setdefault(tuple(p["n"]), []).append(i)
    combo.solve_batch(probs[:6], ctx=ctx, fields=False, precision=prec, tol=1e-8)  # module load, set-up paths
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res_m = combo.solve_batch(probs, ctx=ctx, fields=False, precision=prec, tol=1e-8)
    torch.cuda.synchronize()
    tm = time.perf_counter() - t0
    t0 = time.perf_counter()
    res_b = [None] * len(probs)
    for n, idx in sorted(groups.items()):
        out = combo.solve_batch([probs[i] for i in idx], ctx=ctx, fields=False, precision=prec, tol=1e-8)
        for i, r in zip(idx, out):
            res_b[i] = r
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    t0 = time.perf_counter()
    res_s = [combo.solve(p, ctx=ctx, fields=False, precision=prec, tol=1e-8) for p in probs]
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    vit = sum(int(r["n_operator"]) * int(np.prod(p["n"])) for r, p in zip(res_m, probs))

    def maxrel(xs, ys):
        return max(float(np.max(np.abs(a["Pbar"] - b["Pbar"])) / np.max(np.abs(b["Pbar"]))) for a, b in zip(xs, ys))

    return {"solves": len(probs), "sides": sorted({int(p["n"][0]) for p in probs}), "load_steps": 5,
            "groups": {f"{k[0]}^3": len(v) for k, v in sorted(groups.items())},
            "mixed_seconds": tm, "mixed_solves_per_s": len(probs) / tm, "mixed_voxel_iterations_per_s": vit / tm,
            "per_size_seconds": tb, "per_size_solves_per_s": len(probs) / tb,
            "one_by_one_seconds": ts, "one_by_one_solves_per_s": len(probs) / ts,
            "speedup_mixed_vs_one_by_one": ts / tm, "speedup_per_size_vs_one_by_one": ts / tb,
            "Pbar_rel_diff_mixed_vs_one_by_one_max": maxrel(res_m, res_s),
            "Pbar_rel_diff_per_size_vs_one_by_one_max": maxrel(res_b, res_s),
            "precision": "FP32 Krylov + double-float residual"}


def normals_bench(combo, ctx, stream, peak, peak_kind, cpu=True, reps=20):
    """Coarse-graining with the Sec. 5 normal detection (combo_coarse_grain):
    the paper's 256^3 ball (radius 0.4 L) to 32^3 composite voxels and to
    8 x 16 x 32 boxels, and a 1 GiB image of seeded random balls (radius 24
    voxels, about 20 % inclusion) to 128^3.  Device-resident image, L2
    flushed (a 256 MiB read) before each call, CUDA events on the call's
    stream around the call and (library events) around each launch; median
    of `reps` calls.  The coarse-graining's speed of light is one read of the
    image plus the writes of the phase codes and boxel lists."""
    import torch

    from paper_2204_13624_gb300 import microstructure as ms

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ball = ms.fine_ball_image(256, 0.4)
    work = [("ball_256_to_32^3", ball, (8, 8, 8)), ("ball_256_to_8x16x32", ball, (32, 16, 8)),
            ("spheres_1024_to_128^3", ms.fine_spheres_image((1024, 1024, 1024), 24, 4000, seed=ms.SEED_BASE + 5),
             (8, 8, 8))]
    out = {}
    combo.coarse_grain_profile(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches = 0
    for name, chi, b in work:
        d = torch.from_numpy(chi).cuda()
        for _ in range(3):
            res = combo.coarse_grain(d, b, ctx=ctx)
        calls, kern = [], []
        for _ in range(reps):
            # evict L2 by reading (a written flush buffer would leave dirty
            # lines whose write-back lands in the timed kernels)
            flush.sum()
            e0.record(stream)
            res = combo.coarse_grain(d, b, ctx=ctx)
            e1.record(stream)
            torch.cuda.synchronize()
            calls.append(e0.elapsed_time(e1))
            kern.append(combo.coarse_grain_profile_read())
            launches += 5
        V = int(chi.size)
        nb = int(res[4])
        nc = V // (b[0] * b[1] * b[2])
        ms_call = statistics.median(calls)
        ms_k = [statistics.median(k[i] for k in kern) for i in range(5)]
        ms_kernels = sum(ms_k)
        # speed of light of the whole coarse-graining: the image read once, the
        # phase codes and the boxel lists (index, normal, c+) written once
        alg_all = V + nc + 40 * nb
        # the packing pass reads the image and writes one bit per voxel
        alg_pack = V + V // 8
        gbps_all = alg_all / (ms_kernels / 1e3) / 1e9
        gbps_pack = alg_pack / (ms_k[0] / 1e3) / 1e9
        # end to end from a host image: H2D of the image, D2H of phases and boxels
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        combo.coarse_grain(chi, b, ctx=ctx)
        t_e2e = time.perf_counter() - t0
        out[name] = {"fine": list(chi.shape[::-1]), "boxel": list(b), "coarse_voxels": nc, "boxels": nb,
                     "ms_call": ms_call, "ms_kernels": ms_kernels, "ms_pack": ms_k[0], "ms_slab": ms_k[1],
                     "ms_scan": ms_k[2], "ms_scatter": ms_k[3], "ms_finish": ms_k[4],
                     "fine_voxels_per_s": V / (ms_kernels / 1e3),
                     "fine_voxels_per_s_call": V / (ms_call / 1e3),
                     "roofline": {"bound": "hbm", "achieved": gbps_all, "peak": peak, "unit": "GB/s",
                                  "frac": gbps_all / peak, "peak_kind": peak_kind, "alg_bytes": alg_all,
                                  "what": "all five kernels against one read of the image"},
                     "roofline_pack": {"bound": "hbm", "achieved": gbps_pack, "peak": peak, "unit": "GB/s",
                                       "frac": gbps_pack / peak, "peak_kind": peak_kind, "alg_bytes": alg_pack},
                     "e2e": {"value": V / t_e2e, "unit": "fine voxels/s", "h2d_bytes": V,
                             "d2h_bytes": nc + 40 * nb, "seconds": t_e2e}}
        del d
        if cpu and name == "ball_256_to_32^3":
            from oracle import normals as nrm

            t0 = time.perf_counter()
            nrm.block_normals(chi, b, (1.0, 1.0, 1.0))
            dt = time.perf_counter() - t0
            out[name]["cpu_baseline"] = {"value": V / dt, "unit": "fine voxels/s", "cores": 1, "kind": "oracle",
                                         "sample": "the whole 256^3 image, one pass"}
    combo.coarse_grain_profile(False)
    out["sphere_table1"] = sphere_table1(combo, ctx)
    out["note"] = ("ms_call: events around the whole call (five launches, the count's copy back and the "
                   "call's host synchronisation); ms_pack/slab/scan/scatter/finish: library events around each "
                   "launch; fine_voxels_per_s from their sum")
    out["gpu_launches"] = launches
    return out


def variants_bench(combo, ctx):
    """Solver and discretisation variants on one 128^3 problem (seeded random
    balls, radius 8 voxels, vf 0.2, contrast 10, Fbar_11 = 1.05 in 2 steps,
    tol 1e-8): wall clock of combo_solve from host buffers, operator
    applications, and Pbar against the rotated Newton-CG result."""
    import torch

    from paper_2204_13624_gb300 import microstructure as ms

    p = ms.random_spheres((128, 128, 128), 8.0, 0.2, ms.SEED_BASE + 6, 10.0, np.diag([1.05, 1.0, 1.0]), 2)
    V = 128 ** 3
    runs = [("newton_cg_rotated_refined_df", dict(solver=combo.NEWTON_CG, precision=combo.FP32_REFINED_DF)),
            ("newton_cg_rotated_fp64", dict(solver=combo.NEWTON_CG, precision=combo.FP64)),
            ("newton_cg_spectral_refined_df", dict(solver=combo.NEWTON_CG, precision=combo.FP32_REFINED_DF,
                                                   kspace=combo.SPECTRAL)),
            ("newton_cg_staggered_refined_df", dict(solver=combo.NEWTON_CG, precision=combo.FP32_REFINED_DF,
                                                    kspace=combo.STAGGERED)),
            ("nonlinear_cg_rotated_fp64", dict(solver=combo.NONLINEAR_CG, precision=combo.FP64)),
            ("nonlinear_cg_staggered_fp64", dict(solver=combo.NONLINEAR_CG, precision=combo.FP64,
                                                 kspace=combo.STAGGERED)),
            ("nonlinear_cg_staggered_dfmg_fp64", dict(solver=combo.NONLINEAR_CG, precision=combo.FP64,
                                                      kspace=combo.STAGGERED_DFMG)),
            ("nonlinear_cg_rotated_df", dict(solver=combo.NONLINEAR_CG, precision=combo.FP32_REFINED_DF)),
            ("nonlinear_cg_staggered_dfmg_df", dict(solver=combo.NONLINEAR_CG, precision=combo.FP32_REFINED_DF,
                                                    kspace=combo.STAGGERED_DFMG)),
            ("newton_cg_staggered_dfmg_refined_df", dict(solver=combo.NEWTON_CG, precision=combo.FP32_REFINED_DF,
                                                         kspace=combo.STAGGERED_DFMG)),
            ("newton_cg_staggered_dfmg_fp64", dict(solver=combo.NEWTON_CG, precision=combo.FP64,
                                                   kspace=combo.STAGGERED_DFMG)),
            ("basic_scheme_rotated_fp64", dict(solver=combo.FIXED_POINT, precision=combo.FP64)),
            ("newton_cg_rotated_refined_df_infinitesimal_strain",
             dict(solver=combo.NEWTON_CG, precision=combo.FP32_REFINED_DF, theory=combo.INFINITESIMAL_STRAIN)),
            ("newton_cg_rotated_fp64_infinitesimal_strain",
             dict(solver=combo.NEWTON_CG, precision=combo.FP64, theory=combo.INFINITESIMAL_STRAIN))]
    out = {"problem": "128^3 random balls r=8 vox, vf 0.2, contrast 10, Fbar11 = 1.05 in 2 steps, tol 1e-8"}
    ref = None
    for name, o in runs:
        combo.solve(p, ctx=ctx, fields=False, tol=1e-8, **o)  # warm (tables, autotuner)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = combo.solve(p, ctx=ctx, fields=False, tol=1e-8, **o)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if ref is None:
            ref = r["Pbar"][-1]
        out[name] = {"seconds": dt, "outer_iterations": [int(v) for v in r["iters"]],
                     "operator_applications": int(r["n_operator"]),
                     "voxel_iterations_per_s": int(r["n_operator"]) * V / dt,
                     "Pbar_rel_diff_vs_rotated_newton": float(np.linalg.norm(r["Pbar"][-1] - ref) / np.linalg.norm(ref))}
    out["dfmg_kernels"] = dfmg_kernels(combo, ctx, p)
    out["oracle"] = variants_oracle(combo, p)
    return out


def variants_oracle(combo, p):
    """The oracle beside the variants: one load step of the same 128^3 problem,
    a bounded number of operator applications per variant (FP64, the host
    cores), as voxel-iterations/s."""
    import oracle

    cores = len(os.sched_getaffinity(0))
    V = p["n"][0] * p["n"][1] * p["n"][2]
    runs = [("nonlinear_cg_rotated", dict(solver=2, fixed_iter=2)),
            ("nonlinear_cg_staggered_dfmg", dict(solver=2, kspace=3, fixed_iter=2)),
            ("newton_cg_rotated_infinitesimal_strain", dict(solver=1, theory=1, fixed_iter=1, cg_fixed_iter=4))]
    out = {"cores": cores, "kind": "oracle", "sample": "first load step of the 128^3 problem, FP64"}
    for name, o in runs:
        t0 = time.perf_counter()
        r = oracle.solve(dict(p, n_steps=1), dict(o, nthreads=cores), fields=False)
        dt = time.perf_counter() - t0
        ops = int(r["n_operator"])
        out[name] = {"operator_applications": ops, "seconds": dt, "voxel_iterations_per_s": ops * V / dt}
    return out


def dfmg_kernels(combo, ctx, p):
    """Per-kernel CUDA-event times of the doubly-fine material grid law inside
    a nonlinear-CG solve of the same problem (first load step, 40 iterations
    after 10 untimed).  Algorithmic bytes per cell: dfmg_pure reads F (72 B)
    and writes the 8 sub-cell stresses (576 B); dfmg_gather reads those
    (576 B) and writes P (72 B).  dfmg_pure also does 8 FP64 Neo-Hookean
    evaluations per cell (a logarithm, a division, ~70 FMAs each)."""
    import torch

    n = p["n"]
    V = n[0] * n[1] * n[2]
    out = {"cells": V}
    for form, prec in (("fp64", combo.FP64), ("double_float", combo.FP32_REFINED_DF)):
        out[form] = _dfmg_kernel_times(combo, ctx, p, prec, V)
    return out


def _dfmg_kernel_times(combo, ctx, p, prec, V):
    import torch

    s = combo.Solve(p, ctx=ctx, solver=combo.NONLINEAR_CG, precision=prec, kspace=combo.STAGGERED_DFMG,
                    tol=1e-12)
    s.advance(10)
    torch.cuda.synchronize()
    s.profile(True)
    s.advance(40)
    torch.cuda.synchronize()
    prof = s.profile_read()
    s.profile(False)
    s.close()
    peak, kind = peaks()
    out = {"hbm_peak_gbs": peak, "peak_kind": kind}
    for name, nbytes in (("dfmg_pure", 648), ("dfmg_gather", 648)):
        ms_tot, cnt = prof.get(name, (0.0, 0))
        if cnt:
            per = ms_tot / cnt
            gbs = nbytes * V / (per * 1e-3) / 1e9
            out[name] = {"launches": cnt, "ms_per_launch": per, "algorithmic_GB_s": gbs, "frac_hbm": gbs / peak}
    out["other_kernels_ms_per_iteration"] = {k: v[0] / max(v[1], 1) for k, v in prof.items()
                                             if k not in ("dfmg_pure", "dfmg_gather")}
    return out


def sphere_table1(combo, ctx):
    """Sec. 6.2: Pbar errors (%) of ComBo discretisations of the 256^3 ball
    (Sec. 5 normals and barycentre normals) against the 256^3 rotated-scheme
    reference, beside the paper's printed Table tab:ex:sphere:P1."""
    from paper_2204_13624_gb300 import microstructure as ms

    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "sphere_table1.json")))
    t0 = time.perf_counter()
    ref = combo.solve(ms.sphere_e1_fine(256, 5), ctx=ctx, fields=False, precision=combo.FP32_REFINED_DF, tol=1e-9)
    t_ref = time.perf_counter() - t0
    Pref = ref["Pbar"][-1]
    Pph = ref["Pbar_phase"][-1]
    chi = ms.fine_ball_image(256, 0.4)
    rows = {}
    err = lambda x, y: 100.0 * float(np.linalg.norm(x - y) / np.linalg.norm(y))
    for key, vals in gold["rows"].items():
        b = tuple(256 // int(v) for v in key.split("x"))
        row = {"paper": dict(zip(gold["columns"], vals))}
        for meth, name in (("kabel", "kabel"), ("laplace", "sec5")):
            ph, idx, c, N, nb = combo.coarse_grain(chi, b, method=meth, ctx=ctx)
            r = combo.solve(ms.sphere_e1_coarse(ph, idx, c, N, 5), ctx=ctx, fields=False, precision=combo.FP64,
                            tol=1e-10)
            row[name + "_Pbar"] = err(r["Pbar"][-1], Pref)
            row[name + "_Pbar_matrix"] = err(r["Pbar_phase"][-1][0], Pph[0])
            row[name + "_Pbar_inclusion"] = err(r["Pbar_phase"][-1][1], Pph[1])
            row["boxels"] = int(nb)
        rows[key] = row
    return {"rows": rows, "unit": "% Pbar error", "reference_seconds": t_ref,
            "reference": "256^3 ball, rotated scheme, 5 load steps, refined double-float, tol 1e-9",
            "coarse": "combo_coarse_grain + FP64 ComBo solve, 5 load steps, tol 1e-10"}


def run_reference(args, rank, world):
    """The oracle (FP64 CPU) timed on the host cores.  One oracle CG
    iteration of the full 256^3 grid takes several seconds, so each step is
    one CG operator application of the oracle's Newton-CG (the operation the
    GPU arm's value counts) on a 64^3 RVE of the same microstructure family
    (balls of radius 12 voxels, vf 0.25, contrast 100, Fbar11 = 1.10),
    keeping the whole run within minutes."""
    if rank != 0:
        return
    import oracle
    from paper_2204_13624_gb300 import microstructure as ms

    oracle.build()
    p = ms.random_spheres((64, 64, 64), 12.0, 0.25, ms.SEED_BASE + 1, 100.0, np.diag([1.10, 1.0, 1.0]), 10)
    V = p["n"][0] * p["n"][1] * p["n"][2]
    cores = len(os.sched_getaffinity(0))
    # time of `steps` CG iterations = difference of the two runs (set-up cancels)
    ops, dt, value = oracle_cg_rate(p, max(args.warmup, 1), args.steps, cores, reps=3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(ops, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "64^3 RVE of the spheres_256 family (balls of radius "
                                                      "12 voxels, vf 0.25, contrast 100, Fbar11 = 1.10)",
                       "sample_grid": list(p["n"]), "same_grid_as_gpu_arm": False,
                       "solver": "FP64 oracle Newton-CG, CG operator applications"},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
                             "sample": f"{ops} CG operator applications of the oracle's Newton-CG on a 64^3 RVE "
                                       f"of the {WORKLOAD} family (r = 12 vox balls, vf 0.25, contrast 100); "
                                       "difference of two runs (fastest of 3 each), set-up, residual and "
                                       "laminates cancelled"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
