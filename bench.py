"""Benchmark: forward + adjoint cone-beam projector pair throughput (Gsamples/s).

One step = forward projection P x of a clinical-size phantom followed by the
backprojection P* of that projection (256x256x192 at 2 mm, 400 angles over 360
deg, 512x384 panel at 0.8 mm, +160 mm lateral offset), inputs resident in HBM.
A sample is one (ray, plane) pair of the Joseph sum; a step processes
S_fwd + S_adj = 2 S_fwd samples.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU (torchrun, one rank per GPU): every rank projects its own volume (the
path shards by volume with no data-path collective: weak scaling); the max
over ranks of the timed region is reported.
--impl reference times the FP64 CPU checker (the only reference that exists:
the paper ships no code) on a bounded sample of the same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "clinical"
WORKLOAD_DESC = ("projector pair, 256x256x192 FP32 volume at 2 mm (40 seeded ellipsoids with bone/air inserts), "
                 "400 angles over 360 deg, 512x384 panel at 0.8 mm, +160 mm offset, SID 1000 / SDD 1536 mm")
METRIC = "fwd+adjoint projector Gsamples/s"
L2_BYTES = 129 * 1024 * 1024


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(vals, dist, device):
    """Element-wise maximum of per-rank timings, returned on every rank (the slowest
    rank defines the step time); the values themselves on a single rank."""
    if dist is None:
        return list(vals)
    import torch
    t = torch.tensor(list(vals), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_value(samples_per_rank_step: float, world: int, ms: float) -> float:
    """Gsamples/s of the whole job: every rank projects its own volume (weak scaling),
    so the samples of all ranks over the slowest rank's step time."""
    return samples_per_rank_step * world / (ms * 1e-3) / 1e9


def cpu_reference(steps: int, warmup: int, sample_angles: int, workload: str = WORKLOAD, best: bool = False):
    """FP64 CPU checker on a bounded sample: the workload's geometry restricted to
    `sample_angles` evenly spaced angles (same volume, panel and ray count per
    angle); throughput in Gsamples/s of forward + adjoint (mean of the timed steps,
    or the best one)."""
    import numpy as np

    import oracle as O
    from paper_2512_21180_gb300 import inputs as I

    g = I.geometry(workload)
    ang = 2 * np.pi * np.arange(0, g["n_angles"], g["n_angles"] // sample_angles)[:sample_angles] / g["n_angles"]
    gs = dict(g)
    gs["n_angles"] = len(ang)
    G = O.Geom(gs, angles=ang)
    vol = O.phantom(G, I.phantom_params(workload, 2))
    _, ns = O.forward(G, vol, return_count=True)
    times = []
    for it in range(warmup + steps):
        t0 = time.perf_counter()
        p = O.forward(G, vol)
        O.adjoint(G, p)
        dt = time.perf_counter() - t0
        if it >= warmup:
            times.append(dt)
    mean = min(times) if best else sum(times) / len(times)
    return {"value": 2 * ns / mean / 1e9, "sec_per_step": mean, "samples_per_step": 2 * ns,
            "cores": O.num_threads(), "angles": len(ang)}


def cpu_reference_single_core(sample_angles: int = 1) -> dict:
    """The same FP64 checker restricted to one OpenMP thread (a child process, since
    the thread count is fixed when OpenMP starts), on `sample_angles` clinical angles."""
    import subprocess
    env = dict(os.environ, OMP_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.cpu_reference(1, 0, %d)))" % (os.path.dirname(os.path.abspath(__file__)),
                                                                   sample_angles))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    r = cpu_reference(max(1, args.steps), args.warmup, args.ref_angles)
    sample = (f"{r['angles']} of 400 evenly spaced angles of the clinical workload "
              f"({r['samples_per_step'] / 1e9:.3f} G samples per forward+adjoint step)")
    line = {
        "metric": METRIC, "value": r["value"], "unit": "Gsamples/s", "impl": "reference",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r["sec_per_step"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "sample": sample},
        "cpu_baseline": {"value": r["value"], "unit": "Gsamples/s", "cores": r["cores"], "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": r["value"], "unit": "Gsamples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--ref-angles", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-lpd", action="store_true", help="skip the learned primal-dual vs PDHG timing leg")
    ap.add_argument("--lpd-only", action="store_true", help="run only the learned primal-dual timing leg")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="geometry name from paper_2512_21180_gb300.inputs (profiling runs use smaller ones)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.lpd_only:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_2512_21180_gb300 import build as B
        B.build()
        print(json.dumps(lpd_timing(args.warmup, max(1, args.steps))), flush=True)
        return 0

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2512_21180_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    if dist is not None:
        dist.barrier()
    from paper_2512_21180_gb300 import inputs as I
    from paper_2512_21180_gb300 import projector as P
    from paper_2512_21180_gb300 import ops

    g = I.geometry(args.workload)
    geom = P.Geometry(g)
    S_fwd = geom.count_samples()
    samples_step = 2 * S_fwd
    ell = I.phantom_params(args.workload, 2 + rank)
    vol = ops.phantom(geom, ell).unsqueeze(0)
    proj = torch.empty((1,) + geom.proj_shape, device="cuda")
    back = torch.empty((1,) + geom.vol_shape, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        P.forward_project(geom, vol, out=proj)
        P.back_project(geom, proj, out=back)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # per-kernel timing on the launching stream, L2 flushed between steps (not timed)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    for e0, e1, e2 in ev:
        flush.fill_(1.0)
        e0.record(stream)
        P.forward_project(geom, vol, out=proj)
        e1.record(stream)
        P.back_project(geom, proj, out=back)
        e2.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    t_fwd = [a.elapsed_time(b) for a, b, _ in ev]
    t_adj = [b.elapsed_time(c) for _, b, c in ev]
    ms = sum(f + a for f, a in zip(t_fwd, t_adj)) / args.steps
    ms_fwd, ms_adj = sum(t_fwd) / args.steps, sum(t_adj) / args.steps
    ms, ms_fwd, ms_adj = max_over_ranks([ms, ms_fwd, ms_adj], dist, "cuda")
    value = whole_job_value(samples_step, world, ms)

    # end to end through the public API with host buffers: pinned host volume in,
    # backprojected volume out, copies inside the timed region
    if args.no_e2e:
        ms_e2e = float("nan")
    else:
        ms_e2e = e2e_leg(args, geom, vol, proj, back, stream, dist)
    e2e = whole_job_value(samples_step, world, ms_e2e)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    return report(args, geom, world, S_fwd, samples_step, value, ms, ms_fwd, ms_adj, e2e, clk, g, dist)


def e2e_leg(args, geom, vol, proj, back, stream, dist):
    import torch

    from paper_2512_21180_gb300 import projector as P

    def step():
        P.forward_project(geom, vol, out=proj)
        P.back_project(geom, proj, out=back)

    host_in = vol.cpu().pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    dvol = torch.empty_like(vol)
    for _ in range(2):
        dvol.copy_(host_in, non_blocking=True)
        step()
        host_out.copy_(back, non_blocking=True)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        dvol.copy_(host_in, non_blocking=True)
        P.forward_project(geom, dvol, out=proj)
        P.back_project(geom, proj, out=back)
        host_out.copy_(back, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1) / args.steps
    if dist is not None:
        ms_e2e = max_over_ranks([ms_e2e], dist, "cuda")[0]
    return ms_e2e


def lpd_timing(warmup: int, reps: int, n_test: int = 8) -> dict:
    """The learned reconstruction against FP32 PDHG-TV on the 128^3 / 200-angle /
    256x192 learned workload (Poisson I0 = 1e5), with the committed trained weights:
    seconds per volume of FDK_w + 8 unrolled iterations (BF16 tensor-core blocks) and of
    FDK_w + 100 PDHG iterations, and the comparison at equal PSNR — mean PSNR over the
    full field of view on n_test held-out test phantoms, the fewest PDHG iterations whose
    mean PSNR reaches the learned reconstruction's, and PDHG's time to get there.
    lambda is the one tuned with the weights (on held-out tuning phantoms)."""
    import json as _json
    import math

    import numpy as np
    import torch

    from paper_2512_21180_gb300 import inputs as I
    from paper_2512_21180_gb300 import ops
    from paper_2512_21180_gb300.experiment_lpd import I0, equal_psnr, make_set
    from paper_2512_21180_gb300.lpd import LPD
    from paper_2512_21180_gb300.projector import Geometry

    wdir = os.path.join(ROOT, "paper_2512_21180_gb300", "weights")
    with open(os.path.join(wdir, "lpd128.json")) as f:
        meta = _json.load(f)
    g = I.geometry("lpd128")
    geom = Geometry(g)
    full = (ops.fov(geom) >= 0.5).float()
    model = LPD(geom, n_iter=meta["n_iter"], n_mem=meta.get("n_mem", 5), residual_input=meta["residual_input"],
                reversible=meta.get("reversible", False), lire=meta.get("lire", False), p4=meta.get("p4", False))
    model.set_params(np.load(os.path.join(wdir, meta["file"])))
    if meta.get("perms"):
        model.set_perms(np.asarray(meta["perms"]))
    nP = ops.opnorm(geom, 0.0, 20)
    gam = nP / math.sqrt(12.0)
    nK = ops.opnorm(geom, gam, 20)
    test = make_set(geom, g, range(30_000, 30_000 + n_test), 90_000)
    out = equal_psnr(geom, model, test, full, meta["pdhg_lambda"], gam, 0.99 / nK, 0.99 / nK)
    out["weights"] = meta["file"]
    out["workload"] = (f"128^3 at 4 mm, 200 angles, 256x192 at 1.6 mm, +80 mm offset, I0 = {I0:g}; "
                       f"{meta['n_iter']} iterations, width 32"
                       + (", data-residual channel" if meta["residual_input"] else "")
                       + (", LIRE iteration" if meta.get("lire") else ", reversible" if meta.get("reversible") else "")
                       + (", P4 primal blocks" if meta.get("p4") else ""))
    return out


def poly_timing(geom, name: str, reps: int = 3) -> dict:
    """Polychromatic primary simulation of one volume of the bench workload (Sec. 2.1:
    water-bone split, two projections, ten energy bins of Poisson draws, log
    normalisation), timed with CUDA events after one warm-up call: the whole call and
    its reading kernel alone (the draws), per volume."""
    import torch

    from paper_2512_21180_gb300 import inputs as I
    from paper_2512_21180_gb300 import ops

    E, mw, mb, _ = I.poly_tables()
    I0 = torch.as_tensor(I.poly_intensity(I.geometry(name)), device="cuda")
    mu = ops.phantom(geom, I.phantom_params(name, 7))
    L, y = ops.poly_simulate(geom, mu, I0, E, mw, mb, I.MU_WATER_60, seed=1)
    ops.poly_reading(L, I0, E, mw, mb, seed=2)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t_all, t_read = 0.0, 0.0
    for r in range(reps):
        ev[0].record(st)
        ops.poly_simulate(geom, mu, I0, E, mw, mb, I.MU_WATER_60, seed=10 + r)
        ev[1].record(st)
        ops.poly_reading(L, I0, E, mw, mb, seed=20 + r)
        ev[2].record(st)
        torch.cuda.synchronize()
        t_all += ev[0].elapsed_time(ev[1])
        t_read += ev[1].elapsed_time(ev[2])
    n_draws = L[0, 0].numel() * len(E)
    return {"ms_per_volume": t_all / reps, "ms_reading": t_read / reps, "bins": len(E),
            "gdraws_s": n_draws / (t_read / reps * 1e-3) / 1e9,
            "note": "stand-in attenuation tables and intensity maps; FP64 Poisson draws (inversion / PTRS)"}


def report(args, geom, world, S_fwd, samples_step, value, ms, ms_fwd, ms_adj, e2e, clk, g, dist):
    import numpy as np

    pk, pk_kind = peaks()
    nvox = int(np.prod(geom.vol_shape))
    nray = int(np.prod(geom.proj_shape))
    # dominant kernel: the slower of the pair
    dom = "back_project" if ms_adj >= ms_fwd else "forward_project"
    ms_dom = max(ms_adj, ms_fwd)
    try:
        smem = smem_peak_gbs()
    except Exception as exc:  # noqa: BLE001 (the derived peak stands in)
        smem = {"error": str(exc)[:200]}
    roof = roofline(dom, ms_dom, S_fwd, nvox, nray, pk, pk_kind, clk, smem)
    roof["traffic"] = MEASURED_TRAFFIC.get(args.workload, {}).get(dom)
    roof["ncu_sm_throughput_pct"] = MEASURED_SM_THROUGHPUT_PCT.get(args.workload, {}).get(dom)
    line = {
        "metric": METRIC, "value": value, "unit": "Gsamples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC if args.workload == WORKLOAD else args.workload,
                   "samples_per_step": samples_step,
                   "l2": "flushed between timed steps (256 MiB write, untimed)",
                   "ms_forward": ms_fwd, "ms_adjoint": ms_adj,
                   "gsamples_s_forward": S_fwd / (ms_fwd * 1e-3) / 1e9,
                   "gsamples_s_adjoint": S_fwd / (ms_adj * 1e-3) / 1e9},
        "roofline": roof,
        "e2e": {"value": e2e, "unit": "Gsamples/s", "h2d_bytes_per_step": nvox * 4, "d2h_bytes_per_step": nvox * 4},
        # per step: forward = two plane transposes + the TMA ray kernel; adjoint = ray
        # weighting + segment gather (+ the fixed-order sum of angle parts when split)
        "gpu_launches": launches_per_step(geom) * args.steps,
        "clocks": clk,
    }
    if not args.no_cpu_baseline and world == 1 and args.workload == WORKLOAD:
        r = cpu_reference(1, 0, args.ref_angles)
        line["cpu_baseline"] = {"value": r["value"], "unit": "Gsamples/s", "cores": r["cores"], "kind": "oracle",
                                "sample": f"{r['angles']} of 400 evenly spaced angles of the same workload, "
                                          f"forward + adjoint, FP64, one step"}
        # the same checker on one core, and on the 64^3 / 64-angle operator-test workload
        # (context only: a failure here must not cost the bench line)
        try:
            r1 = cpu_reference_single_core(1)
            line["cpu_baseline"]["single_core"] = {"value": r1["value"], "cores": r1["cores"],
                                                   "sample": "1 of 400 angles of the same workload, one step"}
        except Exception as exc:  # noqa: BLE001
            line["cpu_baseline"]["single_core"] = {"error": str(exc)[:200]}
        try:
            rs = cpu_reference(3, 0, 64, workload="small64", best=True)
            line["cpu_baseline"]["small64"] = {"value": rs["value"], "cores": rs["cores"],
                                               "sample": "64^3 at 4 mm, all 64 angles, 96x64 panel; best of 3"}
        except Exception as exc:  # noqa: BLE001
            line["cpu_baseline"]["small64"] = {"error": str(exc)[:200]}
    if world == 1:
        try:
            line["poly_primary"] = poly_timing(geom, args.workload)
        except Exception as exc:  # noqa: BLE001 (a leg beside the projector metric)
            line["poly_primary"] = {"error": str(exc)[:300]}
    if not args.no_lpd and world == 1 and args.workload == WORKLOAD:
        try:
            line["lpd_vs_pdhg"] = lpd_timing(1, 2)
        except Exception as exc:  # noqa: BLE001 (a leg beside the projector metric)
            line["lpd_vs_pdhg"] = {"error": str(exc)[:300]}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch, from one ncu
# --set full capture of the clinical workload with the current kernels; None elsewhere
# and whenever the kernel changes after the capture.
MEASURED_TRAFFIC = {"clinical": {"back_project": None, "forward_project": 136.448e6 + 280.638e6}}
# The binding on-chip level's throughput from the same captures: the projector kernels are
# bound by SM instruction issue, so this is sm__throughput.avg.pct_of_peak_sustained_elapsed
# (issue active: forward 75.0 %). Same validity rule as the traffic: the adjoint's capture
# (619 MB, 74.0 %) predates its brick-level reach test, so both figures are withheld for it.
MEASURED_SM_THROUGHPUT_PCT = {"clinical": {"back_project": None, "forward_project": 75.0}}


def launches_per_step(geom) -> int:
    """Kernels one forward + adjoint step launches (mirrors the launchers: 3 for the
    staged forward, 2 for the segment gather, +1 when its angles are split)."""
    import torch
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    nx, ny, nz = geom.g["n"]
    bricks = -(-nx // 16) * -(-ny // 16) * -(-nz // 16)
    parts = min(16, max(1, -(-nsm * 9 // bricks)), geom.g["n_angles"])
    return 3 + 2 + (1 if parts > 1 else 0)


def smem_peak_gbs(reps: int = 5) -> dict:
    """Shared-memory read bandwidth measured on this GPU: cbct_smem_probe (152 SMs x 8
    CTAs x 256 threads, conflict-free 16-byte loads), CUDA events on the launching stream,
    best of `reps` after two warm-up launches."""
    import ctypes

    import torch

    from paper_2512_21180_gb300 import _lib
    lib = _lib.load()
    sink = torch.zeros(152 * 8, device="cuda")
    st = torch.cuda.current_stream()
    nbytes = ctypes.c_longlong(0)
    best = None
    for i in range(reps + 2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        _lib.check(lib.cbct_smem_probe(8, 4096, sink.data_ptr(), ctypes.byref(nbytes), st.cuda_stream),
                   "cbct_smem_probe")
        e1.record(st)
        torch.cuda.synchronize()
        if i >= 2:
            gbs = nbytes.value / (e0.elapsed_time(e1) * 1e-3) / 1e9
            best = gbs if best is None else max(best, gbs)
    return {"gbs": best, "bytes_per_launch": nbytes.value}


def roofline(kernel, ms, S_fwd, nvox, nray, pk, pk_kind, clk, smem=None):
    """Roofline of the dominant kernel. The projector is a gather: its algorithmic
    on-chip traffic is 16 B per sample (the four FP32 bilinear neighbours, read from
    shared memory), so the binding unit is the SM's L1/shared-memory datapath. Its peak
    is measured by the shared-memory read probe (smem_peak_gbs); without it, derived
    from the unit count and clock (152 SMs x 128 B/clk x max SM clock)."""
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    achieved = 16.0 * S_fwd / (ms * 1e-3) / 1e9
    if smem and smem.get("gbs"):
        peak = smem["gbs"]
        kind = "measured: shared-memory read probe (152 SM x 8 CTAs x 256 threads, 16 B loads), best of 5"
    else:
        peak = 152 * 128 * sm_mhz * 1e6 / 1e9   # GB/s
        kind = f"derived: L1/SMEM datapath 152 SM x 128 B/clk x {sm_mhz:.0f} MHz"
    return {"kernel": kernel, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None, "peak_kind": kind,
            "derived_peak": 152 * 128 * sm_mhz * 1e6 / 1e9,
            "hbm": {"compulsory_bytes": 4 * (nvox + nray), "peak_gbs": pk.get("hbm_gbs"), "peak_kind": pk_kind}}


if __name__ == "__main__":
    sys.exit(main())
