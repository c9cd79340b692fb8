"""Benchmark of the Hubbard exact-diagonalization hot path on one GB300.

Workload: the 4x4 periodic square lattice (32 bonds), N_up = N_dn = 8
(D = 12870^2 = 1.656e8), t = 1, U = 8, binary64 vectors, seeded
uniform[-1, 1) start vector (SplitMix64, seed 1234).

One timed step is one H*v (hubbard_apply) on inputs resident in HBM; the
vectors (1.3 GB each) are larger than L2, so no flush is needed between
steps.  value = algorithmic bytes / time, with algorithmic bytes per H*v =
2*D*8 (read v, write w) + the per-spin tables.  The same run also times full
ground-state solves (create + Lanczos to rho < 1e-10 + destroy) and reports
solves/s and p50/p99 latency, each solve checked against the stored oracle
energy (1e-9 relative).

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

--impl reference times the CPU oracle (plain-C Kronecker-sum H*v) on the
host cores for the same metric on a bounded sample.  With N > 1 (torchrun)
every rank runs an independent replica (the path does not shard).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "H·v GB/s vs HBM peak; ground-state solves/s, p50/p99 at ≤1e-9 rel"
# name -> (lattice, N_up, N_dn, U, dtype); the first is the benchmarked workload,
# the others are smaller cases of the same kernels for profiling
WORKLOADS = {
    "sq4x4_n8_8_U8_f64": ("sq4x4", 8, 8, 8.0, "f64"),
    "sq4x4_n8_8_U8_f32": ("sq4x4", 8, 8, 8.0, "f32"),
    "sq4x4_n6_6_U8_f64": ("sq4x4", 6, 6, 8.0, "f64"),
    "sq4x4_n6_6_U8_f32": ("sq4x4", 6, 6, 8.0, "f32"),
}
GOLDEN = os.path.join(ROOT, "tests", "golden", "sq4x4_n8_8_U8.json")


def workload_config(name):
    from workload import lattice_by_name
    lat, nup, ndn, U, dt = WORKLOADS[name]
    ns, bonds = lattice_by_name(lat)
    dup, ddn = math.comb(ns, nup), math.comb(ns, ndn)
    s = 8 if dt == "f64" else 4
    cfg = dict(workload=name, lattice=f"{lat} periodic ({len(bonds)} bonds)", nup=nup, ndn=ndn, t=1.0, U=U,
               dim=dup * ddn, vector_bytes=dup * ddn * s, seed=1234,
               l2_policy=("inputs larger than L2 (%.2f GB vectors vs 129 MB L2); no flush" % (dup * ddn * s / 1e9)))
    return ns, bonds, nup, ndn, U, dt, cfg


# DRAM bytes per hubbard_apply from one ncu metrics capture on the bench sector
# itself (dram__bytes_read.sum + dram__bytes_write.sum over the apply's three
# kernels; one replay pass each), with the SHA-256 prefix of the H*v kernel
# sources it was taken on: a figure is reported only while those sources are
# unchanged.
TRAFFIC = {"sq4x4_n8_8_U8_f64": (9.467e9, "e76d3a12eb13f131")}
KERNEL_SOURCES = ("paper_1204_3425_gb300/csrc/hv_phases.cu", "paper_1204_3425_gb300/csrc/row_blocks.cuh",
                  "paper_1204_3425_gb300/csrc/hv_epilogue.cuh")
NOMINAL_HBM_GBS = 7900.0          # HBM3e nominal per GPU (vendor figure)


def kernel_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload):
    """DRAM bytes per apply if captured on the current kernel sources, else None."""
    t = TRAFFIC.get(workload)
    if t is None or t[1] != kernel_sources_hash():
        return None
    return t[0]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def hv_bytes(D, tables_bytes, s=8):
    """Algorithmic bytes of one H*v: read v, write w, read the tables once."""
    return 2 * D * s + tables_bytes


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"], samples=0)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=sorted(reasons), samples=len(sm))


def max_over_ranks(value, device="cpu"):
    """MAX of a per-rank float over the default process group (identity on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(bytes_per_step, steps, total_ms, world):
    """Whole-job GB/s: every rank runs its own replica of the same work."""
    return world * bytes_per_step * steps / (total_ms * 1e-3) / 1e9


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    import paper_1204_3425_gb300 as hub
    from paper_1204_3425_gb300 import build as hbuild
    from workload import square, start_vector

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hbuild.build()
    hub.load_library()
    stream = torch.cuda.current_stream()

    ns, bonds, nup, ndn, U, dts, cfg = workload_config(args.workload)
    tdt = torch.float64 if dts == "f64" else torch.float32
    esize = 8 if dts == "f64" else 4
    H = hub.hubbard_sector_create(ns, bonds, nup, ndn, 1.0, U)
    D = H.D
    tables = sum(int(hub.load_library().hubbard_table_nnz(H.handle, s)) * 4 + (H.Dup if s == 0 else H.Ddn) * 12
                 for s in (0, 1))
    nbytes = hv_bytes(D, tables, esize)
    v_host = torch.from_numpy(start_vector(D, seed=1234)).to(tdt)
    v_host /= v_host.norm()
    v_pin = v_host.pin_memory()
    v = v_pin.to(dev, non_blocking=True)
    w = torch.empty_like(v)
    torch.cuda.synchronize()

    # ---- H*v steps (inputs resident) -------------------------------------
    if args.no_autotune:
        schedule = (0, 0, 0, 0)                             # the library's default choice
    else:
        schedule = hub.hubbard_autotune_schedule(H, v, w)   # fastest (vec_rows, vec_cols, ctas_rows, -)
    for _ in range(args.warmup):
        hub.hubbard_apply(H, v, w)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = hub.hubbard_kernel_launches()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        hub.hubbard_apply(H, v, w)
        ev[i][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = hub.hubbard_kernel_launches() - launches0
    total_ms = t_start.elapsed_time(t_end)
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    per = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(total_ms, dev)
    ms = total_ms / args.steps
    value = job_throughput(nbytes, args.steps, total_ms, ws)

    # ---- end to end through the C ABI with host buffers -------------------
    # every step uploads its input from pinned host memory, applies H and
    # downloads its result; three streams overlap step i+1's upload and step
    # i-1's download with step i's H*v (two device buffers each way)
    e2e_ms = e2e_host_apply(hub, torch, H, v_pin, D, tdt, dev, max(4, min(args.steps, 8)))
    e2e_val = ws * nbytes / (e2e_ms * 1e-3) / 1e9

    # ---- ground-state solves ----------------------------------------------
    golden = json.load(open(GOLDEN))["e0"]
    n_solves = args.solves if args.workload == "sq4x4_n8_8_U8_f64" else 0
    lat, iters, errs, it_times = [], [], [], []
    ws_buf = torch.empty(hub.lanczos_workspace_bytes(H, hub.HUB_F64), dtype=torch.uint8, device=dev)
    v0 = torch.from_numpy(start_vector(D, seed=1234)).to(dev)
    for k in range(n_solves + 1 if n_solves > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Hs = hub.hubbard_sector_create(16, bonds, 8, 8, 1.0, 8.0)
        tc = time.perf_counter()
        r = hub.lanczos_ground_state(Hs, v0, 600, 1e-10, workspace=ws_buf)
        torch.cuda.synchronize()
        t_it = (time.perf_counter() - tc) / max(1, r["iters"])
        Hs.close()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if k == 0:
            continue                     # warm-up solve
        lat.append(dt)
        it_times.append(t_it)
        iters.append(r["iters"])
        errs.append(abs(r["energy"] - golden) / abs(golden))
    ok = [e <= 1e-9 for e in errs]
    solve = dict(solves=n_solves, solves_per_s=sum(ok) / sum(lat) if lat else None,
                 ms_per_iteration=1e3 * float(np.median(it_times)) if it_times else None,
                 p50_ms=1e3 * float(np.percentile(lat, 50)) if lat else None,
                 p99_ms=1e3 * float(np.percentile(lat, 99)) if lat else None,
                 iters=iters, max_rel_err=max(errs) if errs else None, all_within_1e9=all(ok),
                 tol="rho < 1e-10", includes="hubbard_sector_create + lanczos_ground_state + destroy")

    extra = {}
    if args.workload == "sq4x4_n8_8_U8_f64" and args.solves > 0:
        extra["solve_refined"] = bench_refined(hub, torch, dev, bonds, golden, args.solves)
    if args.batch and rank == 0:
        extra["batch"] = bench_batch(hub, torch, dev, count=args.batch_sectors, autotune=not args.no_autotune)
    if args.serve and rank == 0:
        extra["serve"] = bench_serve(args.serve, args.serve_lanes)

    if args.workload == "sq4x4_n8_8_U8_f64":
        extra["hv_sq4x4_f32"] = bench_hv_f32(hub, torch, H, v_host, args.steps, args.warmup)
        if args.evolve:
            extra["time_evolve"] = bench_evolve(hub, torch, dev, H, v,
                                                cpu=(rank == 0 and ws == 1 and not args.no_cpu_baseline))
    H.close()
    del v, w, v_pin
    torch.cuda.empty_cache()
    if args.ring18 and args.workload == "sq4x4_n8_8_U8_f64":
        extra["config3_ring18"] = bench_ring18(hub, torch, dev, args.ring18_U,
                                               cpu=(rank == 0 and ws == 1 and not args.no_cpu_baseline))
    peak, src = peaks()
    avg_kernel_ms = float(np.mean(per))
    achieved = nbytes / (avg_kernel_ms * 1e-3) / 1e9
    traffic = measured_traffic(args.workload)
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dts,
        "arith": ("exact int32-pair fixed-point hop sums, binary64 storage and rounding" if dts == "f64"
                  else "binary32"),
        "data": "synthetic (seeded SplitMix64 start vector)",
        "config": dict(cfg, step="one H*v (hubbard_apply)"),
        "parallelism": "replicas" if ws > 1 else "single",
        "schedule": dict(zip(("vec_rows", "vec_cols", "ctas_rows", "ctas_cols"), schedule)),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_source": src,
                     "algorithmic_bytes_per_launch": nbytes,
                     "frac_of_nominal_7900": achieved / NOMINAL_HBM_GBS,
                     "dram_gbs_from_traffic": (traffic / (avg_kernel_ms * 1e-3) / 1e9 if traffic else None),
                     "dram_frac_from_traffic": (traffic / (avg_kernel_ms * 1e-3) / 1e9 / peak if traffic else None),
                     "amplification": (traffic / nbytes if traffic else None),
                     "kernel_sources_sha": kernel_sources_hash(),
                     "kernel": "hubbard_apply (row phase + up phase kernels)"},
        "e2e": {"value": e2e_val, "unit": "GB/s", "h2d_bytes_per_step": D * esize, "d2h_bytes_per_step": D * esize,
                "ms_per_step": e2e_ms, "api": "hubbard_apply_host (C ABI, page-locked host buffers)",
                "pipelined": "inside the library: upload i+1 | H*v i | download i-1 (two staging slots, three streams)"},
        "gpu_launches": int(launches),
        "clocks": clk,
        "solve": solve,
    }
    line.update(extra)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and args.workload == "sq4x4_n8_8_U8_f64":
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        attach_solve_baselines(line, args.batch_sectors, args.serve, args.cpu_seconds / 2)
    for key in ("batch", "serve"):
        if key in line:
            line[key].pop("_energies", None)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


def e2e_host_apply(hub, torch, H, v_pin, D, tdt, dev, k):
    """ms per step of k hubbard_apply_host calls (the C ABI's host-buffer product:
    page-locked input and output; the library overlaps the upload of call i+1 and
    the download of call i-1 with the H*v of call i).  CUDA events on the caller's
    stream, which waits for every download; the device is idle when t0 is recorded,
    so the first upload starts after it."""
    s = torch.cuda.current_stream()
    wpin = [torch.empty(D, dtype=tdt).pin_memory() for _ in range(2)]
    hub.hubbard_apply_host(H, v_pin, wpin[0], stream=s)      # warm: allocates the staging
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(s)
    for i in range(k):
        hub.hubbard_apply_host(H, v_pin, wpin[i & 1], stream=s)
    t1.record(s)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / k


def time_apply(hub, torch, H, v, w, steps, warmup):
    """Mean CUDA-event time (ms) of `steps` hubbard_apply calls after `warmup` ones."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        hub.hubbard_apply(H, v, w)
    torch.cuda.synchronize()
    per = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hub.hubbard_apply(H, v, w)
        e1.record(stream)
        per.append((e0, e1))
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in per]))


def tables_bytes(hub, H):
    """Per-spin tables read once per H*v: packed targets + sign mask + state word."""
    return sum(int(hub.load_library().hubbard_table_nnz(H.handle, s)) * 4 + (H.Dup if s == 0 else H.Ddn) * 12
               for s in (0, 1))


def hv_line(ms, D, tables, s):
    peak, src = peaks()
    nbytes = hv_bytes(D, tables, s)
    gbs = nbytes / (ms * 1e-3) / 1e9
    return dict(ms=ms, gbs=gbs, algorithmic_bytes=nbytes, roofline={"bound": "hbm", "achieved": gbs, "peak": peak,
                "unit": "GB/s", "frac": gbs / peak, "traffic": None, "peak_source": src})


def bench_hv_f32(hub, torch, H, v_host, steps, warmup):
    """The same sector's H*v with binary32 vectors (the refined path's hot loop)."""
    v = v_host.to(torch.float32).cuda()
    w = torch.empty_like(v)
    ms = time_apply(hub, torch, H, v, w, max(steps, 5), warmup)
    out = hv_line(ms, H.D, tables_bytes(hub, H), 4)
    out["dtype"] = "f32"
    del v, w
    return out


def bench_evolve(hub, torch, dev, H, v, t=0.05, krylov_max=30, tol=1e-10, reps=3, cpu=True):
    """Time propagation exp(-iHt) v of the normalised start vector on the
    bench sector (binary64, Lanczos vectors stored in the workspace), timed
    whole (the call synchronises); one untimed warm-up call."""
    torch.cuda.empty_cache()
    ws = torch.empty(hub.hubbard_evolve_workspace_bytes(H, krylov_max, True), dtype=torch.uint8, device=dev)
    ore, oim = torch.empty_like(v), torch.empty_like(v)
    times, info = [], None
    for k in range(reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, info = hub.hubbard_time_evolve(H, v, None, t, krylov_max=krylov_max, tol=tol, workspace=ws,
                                             out_re=ore, out_im=oim)
        dt = time.perf_counter() - t0
        if k > 0:
            times.append(dt)
    # reversibility: evolving back by -t returns v (a property that holds at any size)
    bre, bim, _ = hub.hubbard_time_evolve(H, ore, oim, -t, krylov_max=krylov_max, tol=tol, workspace=ws)
    back = float(torch.sqrt(torch.sum((bre - v) ** 2) + torch.sum(bim ** 2)))
    del ws, ore, oim, bre, bim
    torch.cuda.empty_cache()
    ms = 1e3 * float(np.median(times))
    # algorithmic bytes: each Lanczos step 3 D s (read f_j, read and write the
    # other vector), the combining pass m + 4 vectors (m stored, both parts
    # read and written; m = krylov_dim, exact for the one-step, one-part call
    # timed here); the copies into the stored basis are not counted
    D8 = H.D * 8
    alg = info["hv"] * 3 * D8 + (info["krylov_dim"] + 4) * D8 * info["steps"]
    peak, src = peaks()
    out = dict(workload="sq4x4_n8_8_U8 exp(-iHt) v, |v| = 1", t=t, krylov_max=krylov_max, tol=tol,
               basis="stored in the workspace", ms=ms, steps=info["steps"], hv=info["hv"],
               krylov_dim=info["krylov_dim"], ms_per_hv=ms / max(1, info["hv"]),
               err_estimate=info["err_estimate"], norm_drift=abs(info["norm"] - 1.0), return_error=back,
               includes="Lanczos steps with the stop test, the tridiagonal QR, the one-pass combination",
               roofline={"bound": "hbm", "achieved": alg / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / (ms * 1e-3) / 1e9 / peak, "traffic": None, "peak_source": src,
                         "algorithmic_bytes_per_call": alg})
    if cpu:
        out["oracle_side_by_side"] = evolve_vs_oracle(hub, torch, dev)
    return out


def evolve_vs_oracle(hub, torch, dev, t=0.25):
    """The oracle's propagation (expm_multiply on the explicit sparse H, host
    cores) beside the GPU on the ring 12 (5,5) U = 4 sector (6.3e5 elements,
    complex start), with their largest difference."""
    from oracle import propagate as pr
    from oracle.basis import Sector
    from workload import lattice_by_name, start_vector
    ns, bonds = lattice_by_name("ring12")
    H = hub.hubbard_sector_create(ns, bonds, 5, 5, 1.0, 4.0)
    vr = torch.from_numpy(start_vector(H.D, seed=21)).to(dev)
    vi = torch.from_numpy(start_vector(H.D, seed=1021)).to(dev)
    times = []
    for k in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ore, oim, info = hub.hubbard_time_evolve(H, vr, vi, t, krylov_max=40, tol=1e-10)
        if k > 0:
            times.append(time.perf_counter() - t0)
    got = ore.cpu().numpy() + 1j * oim.cpu().numpy()
    S = Sector(ns, bonds, 5, 5, 1.0, 4.0)
    v = vr.cpu().numpy() + 1j * vi.cpu().numpy()
    t0 = time.perf_counter()
    want = pr.evolve_sparse(S, v, t)
    cpu_s = time.perf_counter() - t0
    H.close()
    return dict(workload="ring12_n5_5_U4 exp(-iHt) v, complex v, t = 0.25, tol 1e-10", dim=S.D,
                gpu_ms=1e3 * float(np.median(times)), gpu_hv=info["hv"],
                oracle_s=cpu_s, oracle="oracle.propagate.evolve_sparse: explicit sparse H built, then scipy "
                "expm_multiply (host cores; both timed)", max_abs_diff=float(np.abs(got - want).max()),
                norm_v=float(np.linalg.norm(v)))


def bench_ring18(hub, torch, dev, U, cpu=True):
    """Config 3: the 18-site ring, N = (9, 9), D = 2.36e9, t = 1, U: binary32 and
    binary64 H*v, then one plain binary64 ground-state solve and one binary32 +
    binary64-refined solve from the same seeded start vector, each checked
    against the stored oracle energy; one solve per path keeps the run short."""
    from workload import ring
    name = f"ring18_n9_9_U{int(U)}"
    e_ref = json.load(open(os.path.join(ROOT, "tests", "golden", name + ".json")))["e0"]
    bonds = ring(18)
    out = {"workload": name, "dim": 48620 ** 2, "t": 1.0, "U": U, "seed": 1234, "solves_per_path": 1,
           "oracle_energy": f"tests/golden/{name}.json"}
    H = hub.hubbard_sector_create(18, bonds, 9, 9, 1.0, U)
    D = H.D
    tb = tables_bytes(hub, H)
    ws_bytes = hub.lanczos_workspace_bytes(H, hub.HUB_F64)
    v = torch.empty(D, dtype=torch.float64, device=dev)
    hub.hubbard_fill_start_vector(v, 1234)          # the seeded recipe, generated on the device
    w = torch.empty_like(v)
    out["hv_f64"] = hv_line(time_apply(hub, torch, H, v, w, 5, 2), D, tb, 8)
    del w
    v32 = v.to(torch.float32)
    w32 = torch.empty_like(v32)
    out["hv_f32"] = hv_line(time_apply(hub, torch, H, v32, w32, 5, 2), D, tb, 4)
    del v32, w32
    H.close()
    torch.cuda.empty_cache()
    # plain binary64 solve (create + Lanczos to rho < 1e-10 + destroy)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Hs = hub.hubbard_sector_create(18, bonds, 9, 9, 1.0, U)
    r = hub.lanczos_ground_state(Hs, v, 1000, 1e-10, workspace=ws)
    Hs.close()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    rel = abs(r["energy"] - e_ref) / abs(e_ref)
    out["solve_f64"] = dict(s=dt, solves_per_s=(1.0 / dt) if rel <= 1e-9 else 0.0, iters=r["iters"],
                            energy=r["energy"], rel_err_vs_oracle=rel, err_bound=r["err_bound"],
                            ms_per_iteration=1e3 * dt / max(1, r["iters"]))
    del ws
    torch.cuda.empty_cache()
    # binary32 + binary64 refinement; spare workspace stores binary32 Lanczos vectors
    free, _ = torch.cuda.mem_get_info()
    slot = (D * 4 + 255) // 256 * 256
    store = int(max(0, min(128, (free - 40 * D - (8 << 30)) // slot)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Hs = hub.hubbard_sector_create(18, bonds, 9, 9, 1.0, U)
    rr = hub.lanczos_ground_state_refined(Hs, v, 1000, 1e-10, store_vectors=store)
    Hs.close()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    rel = abs(rr["energy"] - e_ref) / abs(e_ref)
    out["solve_refined"] = dict(s=dt, solves_per_s=(1.0 / dt) if rel <= 1e-9 else 0.0,
                                iters_f32_f64=(rr["iters_f32"], rr["iters_f64"]), energy=rr["energy"],
                                rel_err_vs_oracle=rel, error_bound=rr["error_bound"], stored_vectors=store,
                                replayed=rr["replayed"])
    out["refined_over_f64_solves"] = (out["solve_refined"]["solves_per_s"] / out["solve_f64"]["solves_per_s"]
                                      if out["solve_f64"]["solves_per_s"] else None)
    del v
    torch.cuda.empty_cache()
    if cpu:
        out["cpu_baseline"] = ring18_cpu_baseline(U)
    return out


def ring18_cpu_baseline(U):
    """The oracle's Kronecker-sum Lanczos iteration on the 18-site ring, host cores
    (two iterations after one warm-up step: 38 GB of host memory)."""
    from oracle.kron import KronHamiltonian, lanczos_matrix_free, set_threads
    from workload import ring, start_vector
    cores = set_threads(0)
    t0 = time.perf_counter()
    K = KronHamiltonian(18, ring(18), 9, 9, 1.0, U)
    build_s = time.perf_counter() - t0
    x = start_vector(K.D, seed=1234)
    stamps = []
    lanczos_matrix_free(K, x, 3, on_step=lambda j, e, r: stamps.append(time.perf_counter()), inplace=True)
    it_s = float(np.median(np.diff(stamps)))
    del x, K
    return {"value": it_s, "unit": "s per Lanczos iteration", "cores": cores, "kind": "oracle",
            "sample": f"3 matrix-free Lanczos steps on the ring-18 (9,9) sector (plain C Kronecker-sum H*v, "
                      f"OpenMP, {cores} threads), median of the last two; table build {build_s:.1f} s not timed"}


def bench_refined(hub, torch, dev, bonds, golden, n):
    """4x4 (8,8) U=8 solved with binary32 Lanczos + binary64 refinement (same seed)."""
    from workload import start_vector
    v0 = torch.from_numpy(start_vector(12870 * 12870, seed=1234)).to(dev)
    lat, errs, iters = [], [], []
    for k in range(n + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H = hub.hubbard_sector_create(16, bonds, 8, 8, 1.0, 8.0)
        # room for 128 binary32 Lanczos vectors (85 GB): the Ritz vector needs no replay
        r = hub.lanczos_ground_state_refined(H, v0, 1000, 1e-10, store_vectors=128)
        replayed = r["replayed"]
        H.close()
        torch.cuda.synchronize()
        if k == 0:
            continue
        lat.append(time.perf_counter() - t0)
        errs.append(abs(r["energy"] - golden) / abs(golden))
        iters.append((r["iters_f32"], r["iters_f64"]))
    ok = [e <= 1e-9 for e in errs]
    return dict(solves=n, solves_per_s=sum(ok) / sum(lat), p50_ms=1e3 * float(np.percentile(lat, 50)),
                p99_ms=1e3 * float(np.percentile(lat, 99)), iters_f32_f64=iters, max_rel_err=max(errs),
                all_within_1e9=all(ok), ritz_vector="replayed" if replayed else "from stored binary32 vectors",
                path="binary32 Lanczos + Ritz vector + binary64 Rayleigh/polish")


def bench_batch(hub, torch, dev, count=2048, max_iters=1000, tol=1e-10, autotune=True):
    """2048 uneven sectors in one persistent launch; schedule picked by the autotuner."""
    from workload import batch_sectors, lattice_by_name
    reqs = batch_sectors(count, seed=1234)
    specs = []
    for r in reqs:
        ns, bonds = lattice_by_name(r["lattice"])
        specs.append((ns, bonds, r["nup"], r["ndn"], r["t"], r["U"]))
    t0 = time.perf_counter()
    B = hub.Batch(specs)
    create_s = time.perf_counter() - t0
    v0 = torch.zeros(int(B.offsets[-1]), dtype=torch.float64, device=dev)
    for k, (r, sp) in enumerate(zip(reqs, specs)):
        D = math.comb(sp[0], sp[2]) * math.comb(sp[0], sp[3])
        hub.hubbard_fill_start_vector(v0[int(B.offsets[k]):int(B.offsets[k]) + D], r["seed"])
    ws = torch.empty(B.workspace_bytes(max_iters), dtype=torch.uint8, device=dev)
    t0 = time.perf_counter()
    if autotune:
        chosen = B.autotune(v0, max_iters, tol, ws)  # full solves rank the schedules
    else:
        chosen = 16384                              # the library's default threshold
        B.set_schedule(chosen)
    tune_s = time.perf_counter() - t0
    # the solve (two memsets + one cooperative launch) captured once as a CUDA graph, then replayed
    stream = torch.cuda.Stream(device=dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        B.solve_async(v0, max_iters, tol, ws, stream=stream)      # fixes the descriptors before capture
        stream.synchronize()
        with torch.cuda.graph(graph, stream=stream):
            B.solve_async(v0, max_iters, tol, ws, stream=stream)
        graph.replay()                                           # warm replay
        stream.synchronize()
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record(stream)
        graph.replay()
        ev[1].record(stream)
        stream.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    res = B.results(ws, max_iters, stream=stream)
    table = B.schedule_table()
    _, task_ctas = B.get_schedule()
    B.close()
    mode_name = {3: "smem", 2: "rows-staged", 0: "rows-L2"}
    by = {}
    for t in table:
        key = t["path"] if t["path"] == "sweep" else "task-" + mode_name.get(t["mode"], str(t["mode"]))
        by[key] = by.get(key, 0) + t["sectors"]
    schedule_table = dict(shapes=len(table), sectors_by_schedule=by,
                          rows="[D_up, D_dn, W, sectors, path, mode]",
                          table=[[t["Dup"], t["Ddn"], t["W"], t["sectors"], t["path"],
                                  mode_name.get(t["mode"], t["mode"]) if t["path"] == "task" else "staged"]
                                 for t in table])
    ok = sum(1 for r in res if r["status"] == 0)
    return dict(sectors=count, ms=ms, solves_per_s=ok / (ms * 1e-3), converged=ok, elems_per_cta=chosen,
                autotune_s=tune_s, create_s=create_s, iters_total=sum(r["iters"] for r in res),
                schedule_table=schedule_table, task_ctas=task_ctas,
                launches_per_batch=1, timed="CUDA graph replay", tol="rho < 1e-10 max(1,|theta|)",
                _energies=[r["energy"] if r["status"] == 0 else None for r in res])


def bench_serve(n, lanes=8):
    """Poisson trace (mean 500 req/s) of rings 8-16 and 3x3, 3x4, 4x4 sectors through
    the native continuous-batching server (budget: 80 % of the free device memory).
    solves/s counts answered requests; verified_solves_per_s only those whose own
    error bound is within 1e-9 relative."""
    import torch

    from paper_1204_3425_gb300.serve import Request, SolveServer
    from workload import serve_requests
    torch.cuda.empty_cache()
    reqs = [Request(k, s, s["arrival_s"]) for k, s in enumerate(serve_requests(n, rate=500.0, seed=1234))]
    srv = SolveServer(0.0, n_slots=lanes, small_lanes=1, small_max_dim=20_000, mid_max_dim=2_000_000)
    st = srv.run_trace(reqs, timeout=3600)
    srv.stop()
    st["converged"] = sum(1 for r in reqs if r.result and r.result["status"] == 0)
    st["rate_req_per_s"] = 500.0
    st["offered_s"] = max(r.arrival_s for r in reqs)
    st["paths"] = {p: sum(1 for r in reqs if r.path == p) for p in ("batch", "binary64", "refined")}
    st["_energies"] = [r.result["energy"] if r.result and r.result["status"] == 0 else None for r in reqs]
    return st


def cpu_baseline(budget_s=15.0):
    """The oracle's plain-C Kronecker H*v on this host's cores, bounded sample."""
    from oracle.kron import KronHamiltonian
    from workload import square, start_vector
    t0 = time.perf_counter()
    K = KronHamiltonian(16, square(4, 4), 8, 8, 1.0, 8.0)
    build_s = time.perf_counter() - t0
    x = start_vector(K.D, seed=1234)
    y = np.zeros(K.D)
    tables = sum(len(tg) * 4 + len(st) * 12 for (st, rp, tg, _) in K.tables)
    nbytes = hv_bytes(K.D, tables)
    K.hv_acc(x, y)                                   # warm-up
    times = []
    t_begin = time.perf_counter()
    while time.perf_counter() - t_begin < budget_s or len(times) < 2:
        t1 = time.perf_counter()
        K.hv_acc(x, y)
        times.append(time.perf_counter() - t1)
    per = float(np.median(times))
    # the paper's own setup: one thread (two calls)
    from oracle.kron import set_threads
    prev = set_threads(1)
    t1s = []
    for _ in range(2):
        t1 = time.perf_counter()
        K.hv_acc(x, y)
        t1s.append(time.perf_counter() - t1)
    set_threads(prev)
    per1 = float(np.median(t1s))
    # the paper's CPU metric: time per Lanczos iteration (median of 5 after one warm-up step)
    from oracle.kron import lanczos_matrix_free
    stamps = []
    lanczos_matrix_free(K, x.copy(), 6, on_step=lambda j, e, r: stamps.append(time.perf_counter()), inplace=True)
    it_s = float(np.median(np.diff(stamps)))
    return {"value": nbytes / per / 1e9, "unit": "GB/s", "cores": prev, "kind": "oracle",
            "sample": f"{len(times)} Kronecker-sum H*v calls on the 4x4 (8,8) sector (plain C, OpenMP, "
                      f"{prev} threads), median {per:.3f} s each; table build {build_s:.1f} s not timed",
            "value_1_thread": nbytes / per1 / 1e9, "hv_s_1_thread": per1, "hv_s": per,
            "lanczos_iteration_s": it_s}


def solves_cpu_baseline(kind, count, budget_s):
    """The oracle's matrix-free Lanczos (plain-C Kronecker-sum H*v, OpenMP) over the
    same request list, one request after another in list order, until budget_s of
    solving is spent (the request running at the deadline finishes); table builds
    are not timed, as the GPU figures exclude sector creation."""
    from oracle.kron import KronHamiltonian, lanczos_matrix_free, set_threads
    from workload import batch_sectors, lattice_by_name, serve_requests, start_vector
    reqs = batch_sectors(count, seed=1234) if kind == "batch" else serve_requests(count, rate=500.0, seed=1234)
    cores = set_threads(0)
    solve_s, n, elems, iters, energies = 0.0, 0, 0, 0, []
    while n < len(reqs) and (n == 0 or solve_s < budget_s):
        r = reqs[n]
        ns, bonds = lattice_by_name(r["lattice"])
        K = KronHamiltonian(ns, bonds, r["nup"], r["ndn"], r["t"], r["U"])
        v0 = start_vector(K.D, seed=r["seed"])
        t0 = time.perf_counter()
        res = lanczos_matrix_free(K, v0, min(K.D, 1000), tol=1e-10, inplace=True)
        solve_s += time.perf_counter() - t0
        n, elems, iters = n + 1, elems + K.D, iters + res["iters"]
        energies.append(res["energy"])
    return {"value": n / solve_s, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"the first {n} of the {len(reqs)} {kind} requests in list order ({elems} elements, "
                      f"{iters} Lanczos steps to rho < 1e-10), one after another; {solve_s:.1f} s of solving "
                      f"on {cores} OpenMP threads", "_energies": energies}


def attach_solve_baselines(line, batch_count, serve_count, budget_s):
    """The batch and serving CPU baselines, each with the agreement of the
    oracle's energies and the GPU's on the requests the oracle solved."""
    for key, count in (("batch", batch_count), ("serve", serve_count)):
        if key in line:
            cb = solves_cpu_baseline(key, count, budget_s)
            cb["max_rel_diff_vs_gpu"], cb["compared"] = agreement(line[key].get("_energies", []),
                                                                  cb.pop("_energies"))
            line[key]["cpu_baseline"] = cb


def agreement(gpu, oracle):
    """Largest relative difference |E_gpu - E_oracle| / |E_oracle| over the
    requests both solved (lists in request order; pairs with E_oracle = 0 are
    compared absolutely), and how many were compared."""
    pairs = [(g, o) for g, o in zip(gpu, oracle) if g is not None and o is not None]
    if not pairs:
        return None, 0
    return max(abs(g - o) / abs(o) if o != 0.0 else abs(g - o) for g, o in pairs), len(pairs)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle.kron import KronHamiltonian
    from workload import square, start_vector
    K = KronHamiltonian(16, square(4, 4), 8, 8, 1.0, 8.0)
    x = start_vector(K.D, seed=1234)
    x /= np.linalg.norm(x)
    y = np.zeros(K.D)
    tables = sum(len(tg) * 4 + len(st) * 12 for (st, rp, tg, _) in K.tables)
    nbytes = hv_bytes(K.D, tables)
    for _ in range(args.warmup):
        K.hv_acc(x, y)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        y[:] = 0.0
        K.hv_acc(x, y)
    dt = time.perf_counter() - t0
    value = nbytes * args.steps / dt / 1e9
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SplitMix64 start vector)",
            "config": dict(workload_config("sq4x4_n8_8_U8_f64")[-1], step="one H*v (oracle Kronecker-sum, host cores)"),
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full H*v calls on the 4x4 (8,8) sector"},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="sq4x4_n8_8_U8_f64")
    ap.add_argument("--solves", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="time the default H*v schedule and batch threshold (profiling commands use it: "
                         "no tuning launches)")
    ap.add_argument("--batch", type=int, default=1, help="also time the 2048-sector batched solve (0: skip)")
    ap.add_argument("--batch-sectors", type=int, default=2048,
                    help="sectors in the batched solve (smaller: the profiling case)")
    ap.add_argument("--serve", type=int, default=2000, help="requests in the serving trace (0: skip)")
    ap.add_argument("--serve-lanes", type=int, default=8, help="big lanes of the server")
    ap.add_argument("--ring18", type=int, default=1, help="also time config 3, the 18-site ring (0: skip)")
    ap.add_argument("--evolve", type=int, default=1, help="also time exp(-iHt) v on the bench sector (0: skip)")
    ap.add_argument("--ring18-U", type=float, default=4.0, choices=[2.0, 4.0, 8.0])
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
