"""Throughput of the full ADER-WENO-CT step on one GB300 (zone-updates/s).

Workload (default): cubed-sphere mesh 6 x 64 x 64 angular zones x 64 log shells
in r in [1, 2] (1,572,864 zones), 4th order, FP64, smooth test problem
(rho = 1 + 0.1 sin(2 pi (x+y+z)/sqrt3), p = 1, v = (.5,.5,.5), B = curl of
A = 0.1 (sin 2 pi z, sin 2 pi x, sin 2 pi y)), dt from CFL 0.4 of the initial state;
the FP32-bulk form of the same workload is timed beside it ("fp32_bulk"), and the
6 x 32 x 32 x 32 (196,608 zones) 3rd-order smooth test in both forms as an extra
key ("order3_196608").

Timed region: K steps, each bracketed by CUDA events on the mesh stream, with an
L2 flush (a 512 MB device write) between steps outside the events.  `value` is
zone-updates/s with the state resident in HBM; `e2e` is the same metric through
the C ABI with host (pinned) buffers: upload, step, download every step.

--impl reference times the FP64 CPU oracle (the test oracle, as it stands) on a
bounded sample of the same workload and prints the same JSON line.
Multi-GPU: the path is not sharded in this version ("replicas only"): each rank
runs an independent replica; value = sum over ranks.
"""
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

METRIC = "zone-updates/s per full ADER-WENO-CT step (FP64 vs FP32-bulk), % roofline"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--nr", type=int, default=64)
    ap.add_argument("--order", type=int, default=4)
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the extra 196,608-zone order-3 measurement")
    ap.add_argument("--cfl", type=float, default=0.4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32-bulk measurement")
    ap.add_argument("--compare-steps", type=int, default=10)
    ap.add_argument("--problem", default="smooth",
                    choices=["smooth", "blast", "lowbeta", "sod", "briowu", "ryujones"],
                    help="workload; the spherical shock tubes use their own shells (inputs.DOMAINS)")
    ap.add_argument("--noise", type=float, default=0.0, help="seeded relative density noise")
    ap.add_argument("--positivity", action="store_true")
    ap.add_argument("--riemann", default="hll", choices=["hll", "hlld"], help="face Riemann solver")
    ap.add_argument("--fp32-only", action="store_true", help="time only the FP32-bulk form")
    ap.add_argument("--cfl-every-step", action="store_true",
                    help="device CFL reduction before every timed step (dt read back each step)")
    ap.add_argument("--nq-zone", type=int, default=0, help="cubature points per direction for the initial data")
    ap.add_argument("--nq-edge", type=int, default=8, help="Gauss points per edge for the initial face fluxes")
    ap.add_argument("--adjoint", default="",
                    help="differentiation workload: comma-separated window lengths K (e.g. 1,8,64)")
    ap.add_argument("--fd-directions", type=int, default=16)
    ap.add_argument("--fd-eps", default="1e-6",
                    help="comma-separated central-difference steps (the first is the configured one)")
    ap.add_argument("--convergence", default="",
                    help="order study on the exact entropy wave: comma-separated subdivisions (nr = n)")
    ap.add_argument("--orders", default="2,3,4")
    ap.add_argument("--t-end", type=float, default=0.1)
    ap.add_argument("--shell", default="1.3,1.7", help="radius band of the error norm")
    ap.add_argument("--predictor", type=int, default=None, choices=[0, 1, 2],
                    help="predictor schedule: 0 one thread per zone, 1 one thread per node, 2 the node team "
                         "with the contraction in the variable layout (default: the library's)")
    ap.add_argument("--prism", action="store_true",
                    help="time the ADER-CG predictor on the paper's prism zones (geo_prism_predictor) on "
                         "--prism-zones seeded synthetic frustums at --order")
    ap.add_argument("--prism-zones", type=int, default=1 << 20)
    ap.add_argument("--contraction", action="store_true",
                    help="time the predictor's derivative contraction alone (FP32, CUDA-core and tensor-core "
                         "forms) beside the FP32-bulk predictor kernel on the same workload")
    ap.add_argument("--sample-n", type=int, default=4)
    ap.add_argument("--sample-nr", type=int, default=4)
    return ap.parse_args()


def workload_name(a):
    form = "FP32-bulk" if getattr(a, "fp32_only", False) else "FP64"
    extra = ""
    if getattr(a, "positivity", False):
        extra += ", positivity on"
    if getattr(a, "noise", 0.0):
        extra += ", density noise %g" % a.noise
    if getattr(a, "cfl_every_step", False):
        extra += ", device CFL every step"
    if getattr(a, "riemann", "hll") == "hlld":
        extra += ", HLLD faces"
    return "cubed-sphere %dx%dx%d x %d shells (%d zones), order %d, %s, %s test%s" % (
        6, a.n, a.n, a.nr, 6 * a.n * a.n * a.nr, a.order, form, getattr(a, "problem", "smooth"), extra)


def default_schedule(order, fp32=False):
    """The library's default predictor schedule: the variable-layout team at
    orders 2 and 3 and for the FP32-bulk form, the node team for FP64 at order 4."""
    return 2 if (order <= 3 or fp32) else 1


def kernel_name(stage, pred, positivity=False, order=4, fp32=False):
    """Name of the kernel that runs a stage (the predictor stage has three
    schedules; the variable-layout one runs the node team when positivity is on)."""
    name = "k_" + stage
    if stage == "ader":
        if pred is None:
            pred = default_schedule(order, fp32)
        if pred == 2 and not positivity:
            name += "_vt"
        elif pred != 0:
            name += "_team"
    return name


def sched_name(pred, order, fp32=False):
    """Predictor schedule in use."""
    if pred is None:
        pred = default_schedule(order, fp32)
    return {0: "zone-thread", 1: "node-team", 2: "variable-team"}[pred]


def max_over_ranks(x, ws, device):
    """The largest of the ranks' values of x (the slowest replica's time); x itself
    for one rank."""
    if ws <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.item()


def replica_throughput(zones, steps, t_ms, ws):
    """Whole-job zone-updates/s of ws independent replicas of `zones` zones that all
    ran `steps` steps, the slowest taking t_ms."""
    return ws * zones * steps / (t_ms * 1e-3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
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
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ----------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, %(root)r)
from oracle.step import Oracle
from paper_1905_02504_gb300.inputs import domain, make_problem
pr = make_problem(%(problem)r, noise=%(noise)r)
o = Oracle(%(n)d, %(nr)d, *domain(%(problem)r), %(p)d, gamma=pr.gamma, positivity=%(pos)r)
U, phi = o.initial_state(pr)
dt = o.cfl_dt(U, %(cfl)r)
times = []
for s in range(%(steps)d):
    t0 = time.perf_counter()
    U, phi = o.step(U, phi, dt)
    times.append(time.perf_counter() - t0)
print(json.dumps({"Z": o.mesh.Z, "times": times}))
"""


def oracle_procs():
    """Host cores the oracle baseline uses: one single-threaded oracle process per
    core (the machine's cores, at most 16)."""
    return max(1, min(os.cpu_count() or 1, 16))


def run_oracle(n, nr, p, cfl, steps, problem="smooth", noise=0.0, pos=False, procs=1):
    """Runs procs copies of the oracle sample at once, each single-threaded; returns
    the zones of one copy, each copy's per-step times and the wall-clock span of
    the timed steps of all copies together (mesh setup excluded)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    code = ORACLE_SNIPPET % dict(root=ROOT, n=n, nr=nr, p=p, cfl=cfl, steps=steps, problem=problem,
                                 noise=noise, pos=bool(pos))
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                           text=True, env=env) for _ in range(procs)]
    res = []
    for pr in ps:
        out, err = pr.communicate(timeout=3000)
        if pr.returncode != 0:
            raise RuntimeError("oracle run failed: " + err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    return res


def oracle_throughput(res, skip):
    """Zone-updates per second of all copies: each copy's timed steps run in parallel,
    so the slowest copy's time bounds the span."""
    Z = res[0]["Z"]
    nsteps = len(res[0]["times"]) - skip
    span = max(sum(r["times"][skip:]) for r in res)
    return len(res) * Z * nsteps / span, span / nsteps, Z


def cpu_baseline(a):
    procs = oracle_procs()
    res = run_oracle(a.sample_n, a.sample_nr, a.order, a.cfl, 1, a.problem, a.noise, a.positivity, procs)
    value, _, Z = oracle_throughput(res, 0)
    single = Z / sum(res[0]["times"])
    return {"value": value, "unit": "zone-updates/s", "cores": procs, "kind": "oracle",
            "single_thread_value": single,
            "sample": "1 FP64 oracle step of the same order-%d %s test on the 6x%dx%dx%d mesh (%d zones) "
                      "in each of %d concurrent single-threaded processes, mesh setup excluded" % (
                          a.order, a.problem, a.sample_n, a.sample_n, a.sample_nr, Z, procs)}


def reference_arm(a):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    procs = oracle_procs()
    res = run_oracle(a.sample_n, a.sample_nr, a.order, a.cfl, a.warmup + a.steps, a.problem, a.noise,
                     a.positivity, procs)
    value, step_s, Z = oracle_throughput(res, a.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "zone-updates/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * step_s, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "sample_zones": Z, "copies": procs},
        "cpu_baseline": {"value": value, "unit": "zone-updates/s", "cores": procs, "kind": "oracle",
                         "sample": "each step: one FP64 oracle step of the order-%d %s test on the "
                                   "6x%dx%dx%d mesh (%d zones) in each of %d concurrent single-threaded "
                                   "processes" % (a.order, a.problem, a.sample_n, a.sample_n, a.sample_nr,
                                                  Z, procs)},
        "e2e": {"value": value, "unit": "zone-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


PREDICTOR_SOURCES = ("device.cuh", "mhd_device.cuh", "ader_vt.cuh")


def predictor_fingerprint():
    """sha256 prefix of the predictor kernels' source: the node-team section of
    kernels.cu (from the team sizes to the face-flux stage), ader_vt.cuh, the
    device headers they use and the generator of the compiled pattern
    (refpattern.py, whose row groups set the variable team's work split).
    Edits elsewhere in the library leave it unchanged."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1905_02504_gb300", "csrc")
    k = open(os.path.join(csrc, "kernels.cu")).read()
    a = k.index("template <int P> struct Team;")
    b = k.index("// a4: face fluxes")
    h = hashlib.sha256(k[a:b].encode())
    for f in PREDICTOR_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    h.update(open(os.path.join(ROOT, "paper_1905_02504_gb300", "refpattern.py"), "rb").read())
    return h.hexdigest()[:16]


def captured_traffic(a, kernel, Z, prec="fp64"):
    """DRAM bytes of one launch of the dominant kernel: the DRAM bytes per zone of
    the committed ncu capture of the same kernel, order and form
    (profiles/k_ader_traffic.json; captured on a 196,608-zone case, the traffic
    growing in proportion to the zones) times the zones of this launch; None when
    there is no such capture or the predictor source changed since."""
    try:
        recs = json.load(open(os.path.join(ROOT, "profiles", "k_ader_traffic.json")))["records"]
        fp = predictor_fingerprint()
        for r in recs:
            if (r["kernel"], r["order"], r["form"], r["source_fingerprint"]) == (kernel, a.order, prec, fp):
                return r["dram_bytes_per_zone"] * Z
    except (OSError, KeyError, ValueError):
        pass
    return None


def fp32_bulk_leg(a, mesh64, U0, phi0, dt, stream, flush, barrier, ws):
    """The FP32-bulk form on the same workload: throughput over the same timed
    protocol, roofline of its dominant kernel against the FP32 ALU peak, and its
    per-variable relative L1 error against the FP64 form after the same steps
    from the same initial state (the FP64 form matches the oracle to 1e-12)."""
    import numpy as np
    import torch
    from paper_1905_02504_gb300 import geomhd
    sid = stream.cuda_stream
    from paper_1905_02504_gb300.inputs import domain, make_problem
    m32 = geomhd.Mesh(a.n, a.nr, *domain(a.problem), a.order, prec=geomhd.GEO_FP32_BULK, stream=sid,
                      gamma=make_problem(a.problem).gamma)
    if a.predictor is not None:
        geomhd.geo_set_predictor(m32.h, a.predictor)
    if a.positivity:
        geomhd.geo_set_positivity(m32.h, 1)
    if a.riemann == "hlld":
        geomhd.geo_set_riemann(m32.h, geomhd.GEO_RIEMANN_HLLD)
    m32.upload(U0, phi0)
    with torch.cuda.stream(stream):
        for _ in range(a.warmup):
            m32.step(dt)
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    geomhd.geo_set_stage_timing(m32.h, 1)
    barrier()
    with torch.cuda.stream(stream):
        for i in range(a.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            m32.step(dt)
            ev[i][1].record(stream)
    barrier()
    t_ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in ev), ws, "cuda")
    geomhd.geo_set_stage_timing(m32.h, 0)
    stage_ms, stage_cnt = geomhd.geo_get_stage_timing(m32.h)
    avg = stage_ms / np.maximum(stage_cnt, 1)
    top = int(np.argmax(avg))
    flops, units = geomhd.geo_stage_flops(m32.h)
    achieved = flops[top] * units[top] / (avg[top] * 1e-3) / 1e12
    fp32_probe = geomhd.geo_probe_fma_peak(1, sid) / 1e12
    nominal_fp32 = 152 * 128 * 2 * 2.07e9 / 1e12
    # error against the FP64 form after the same number of steps
    mesh64.upload(U0, phi0)
    m32.upload(U0, phi0)
    for _ in range(a.compare_steps):
        mesh64.step(dt)
        m32.step(dt)
    U64, p64 = mesh64.download()
    U32, p32 = m32.download()
    err = [float(np.abs(U32[v] - U64[v]).sum() / np.abs(U64[v]).sum()) for v in range(8)]
    errp = float(np.abs(p32 - p64).sum() / np.abs(p64).sum())
    _, r32 = m32.divB()
    out = {
        "value": replica_throughput(m32.Z, a.steps, t_ms, ws), "unit": "zone-updates/s",
        "ms_per_step": t_ms / a.steps, "dtype": "f32 bulk / f64 accumulation and updates",
        "roofline": {"bound": "alu", "achieved": achieved, "peak": nominal_fp32, "unit": "TFLOP/s",
                     "frac": achieved / nominal_fp32,
                     "traffic": captured_traffic(a, kernel_name(geomhd.STAGES[top], a.predictor, a.positivity, a.order, True), m32.Z,
                                                "fp32"),
                     "kernel": kernel_name(geomhd.STAGES[top], a.predictor, a.positivity, a.order, True),
                     "peak_kind": "nominal GB300 FP32 (152 SMs x 128 FMA/clk x 2.07 GHz); measured FP32 "
                                  "FMA-chain probe %.1f TFLOP/s" % fp32_probe,
                     "measured_fp32_fma_tflops": fp32_probe},
        "stages": {geomhd.STAGES[s]: {"avg_ms": float(avg[s]), "share": float(stage_ms[s] / stage_ms.sum())}
                   for s in range(geomhd.N_STAGES)},
        "rel_l1_vs_fp64": err, "rel_l1_phi_vs_fp64": errp, "steps_compared": a.compare_steps,
        "predictor": sched_name(a.predictor, a.order, True),
        "divB_rel": r32,
    }
    m32.close()
    return out


def extra_workload(a, stream, flush, barrier, ws, n=32, nr=32, order=3):
    """The 6 x 32 x 32 x 32 (196,608 zones) order-3 smooth test, both forms, with the
    same timed protocol (warm-up, L2 flush between steps, CUDA events on the mesh
    stream): zone-updates/s and ms per step."""
    import torch
    from paper_1905_02504_gb300 import geomhd
    from paper_1905_02504_gb300.inputs import make_problem
    out = {"workload": "cubed-sphere 6x%dx%dx%d x %d shells (%d zones), order %d, smooth test" % (
        n, n, n, nr, 6 * n * n * nr, order, )}
    U0 = phi0 = dt = None
    for key, prec in (("f64", geomhd.GEO_FP64), ("f32_bulk", geomhd.GEO_FP32_BULK)):
        m = geomhd.Mesh(n, nr, 1.0, 2.0, order, prec=prec, stream=stream.cuda_stream)
        if U0 is None:
            U0, phi0 = m.initial_state(make_problem("smooth"))
        m.upload(U0, phi0)
        if dt is None:
            dt = m.cfl_dt(a.cfl)
        with torch.cuda.stream(stream):
            for _ in range(a.warmup):
                m.step(dt)
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(a.steps)]
        with torch.cuda.stream(stream):
            for i in range(a.steps):
                flush.fill_(float(i))
                ev[i][0].record(stream)
                m.step(dt)
                ev[i][1].record(stream)
        barrier()
        t_ms = max_over_ranks(sum(s_.elapsed_time(e) for s_, e in ev), ws, "cuda")
        out[key] = {"value": replica_throughput(m.Z, a.steps, t_ms, ws), "unit": "zone-updates/s",
                    "ms_per_step": t_ms / a.steps}
        m.close()
    return out


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def gpu_arm(a):
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1905_02504_gb300 import geomhd
    from paper_1905_02504_gb300.inputs import make_problem

    stream = torch.cuda.Stream()
    sid = stream.cuda_stream
    prec = geomhd.GEO_FP32_BULK if a.fp32_only else geomhd.GEO_FP64
    from paper_1905_02504_gb300.inputs import domain
    mesh = geomhd.Mesh(a.n, a.nr, *domain(a.problem), a.order, prec=prec, stream=sid,
                       gamma=make_problem(a.problem).gamma)
    if a.predictor is not None:
        geomhd.geo_set_predictor(mesh.h, a.predictor)
    if a.positivity:
        geomhd.geo_set_positivity(mesh.h, 1)
    if a.riemann == "hlld":
        geomhd.geo_set_riemann(mesh.h, geomhd.GEO_RIEMANN_HLLD)
    U0, phi0 = mesh.initial_state(make_problem(a.problem, noise=a.noise), nq_zone=a.nq_zone or None,
                                  nq_edge=a.nq_edge)
    mesh.upload(U0, phi0)
    dt = mesh.cfl_dt(a.cfl)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        for _ in range(a.warmup):
            mesh.step(dt)
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    geomhd.geo_set_stage_timing(mesh.h, 1)
    clk = ClockSampler(local)
    clk.start()
    barrier()
    with torch.cuda.stream(stream):
        for i in range(a.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            if a.cfl_every_step:
                dt = mesh.cfl_dt(a.cfl)
            mesh.step(dt)
            ev[i][1].record(stream)
    barrier()
    clocks = clk.stop()
    step_ms = [s.elapsed_time(e) for s, e in ev]
    geomhd.geo_set_stage_timing(mesh.h, 0)
    stage_ms, stage_cnt = geomhd.geo_get_stage_timing(mesh.h)
    t_ms = max_over_ranks(sum(step_ms), ws, "cuda")
    Z = mesh.Z
    value = replica_throughput(Z, a.steps, t_ms, ws)
    a_div, r_div = mesh.divB()

    # ---- end to end through the C ABI with pinned host buffers
    Uh = torch.from_numpy(U0).pin_memory()
    ph = torch.from_numpy(phi0).pin_memory()
    Uo = torch.empty_like(Uh).pin_memory()
    po = torch.empty_like(ph).pin_memory()
    e2e_steps = max(3, min(a.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        geomhd.geo_state_upload(mesh.h, Uh, ph)
        mesh.step(dt)
        geomhd.geo_state_download(mesh.h, Uo, po)
    barrier()
    t_e2e = time.perf_counter() - t0
    e2e_value = ws * Z * e2e_steps / t_e2e
    finite = bool(torch.isfinite(Uo).all().item() and torch.isfinite(po).all().item())
    bytes_state = (Uh.numel() + ph.numel()) * 8

    # ---- roofline of the dominant kernel (plain FP64 ALU work)
    flops, units = geomhd.geo_stage_flops(mesh.h)
    avg = stage_ms / np.maximum(stage_cnt, 1)
    top = int(np.argmax(avg))
    achieved = flops[top] * units[top] / (avg[top] * 1e-3) / 1e12
    if a.fp32_only:
        fma_peak = geomhd.geo_probe_fma_peak(1, sid) / 1e12
        nominal = 152 * 128 * 2 * 2.07e9 / 1e12
        kind = ("nominal GB300 FP32 (152 SMs x 128 FMA/clk x 2.07 GHz); measured FP32 FMA-chain probe "
                "%.1f TFLOP/s" % fma_peak)
    else:
        fma_peak = geomhd.geo_probe_fma_peak(0, sid) / 1e12
        nominal = 1.25
        kind = "nominal GB300 FP64 (recipe); measured FP64 FMA-chain probe %.3f TFLOP/s" % fma_peak
    roofline = {"bound": "alu", "achieved": achieved, "peak": nominal, "unit": "TFLOP/s",
                "frac": achieved / nominal,
                "traffic": captured_traffic(a, kernel_name(geomhd.STAGES[top], a.predictor, a.positivity, a.order,
                                                           a.fp32_only), Z,
                                            "fp32" if a.fp32_only else "fp64"),
                "kernel": kernel_name(geomhd.STAGES[top], a.predictor, a.positivity, a.order, a.fp32_only),
                "peak_kind": kind, "measured_fma_tflops": fma_peak}
    stages = {geomhd.STAGES[s]: {"avg_ms": float(avg[s]), "share": float(stage_ms[s] / stage_ms.sum())}
              for s in range(geomhd.N_STAGES)}
    fp32 = None if (a.no_fp32 or a.fp32_only) else fp32_bulk_leg(a, mesh, U0, phi0, dt, stream, flush, barrier, ws)
    extra = None if a.no_extra else extra_workload(a, stream, flush, barrier, ws)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "zone-updates/s", "n_gpus": ws,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32-bulk" if a.fp32_only else "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(a), "zones": Z, "order": a.order, "dt": dt,
                       "problem": a.problem, "positivity": a.positivity,
                       "predictor": sched_name(a.predictor, a.order, a.fp32_only),
                       "cfl": a.cfl, "l2": "flushed between steps (512 MB write)",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            # per step: the seven stage kernels, the trace positivity kernel when the
            # limiter is on, the two-kernel CFL reduction when dt is recomputed
            "gpu_launches": int((geomhd.N_STAGES + int(a.positivity) + 2 * int(a.cfl_every_step)) * a.steps),
            "e2e": {"value": e2e_value, "unit": "zone-updates/s", "h2d_bytes_per_step": bytes_state,
                    "d2h_bytes_per_step": bytes_state},
            "roofline": roofline,
            "stages": stages,
            "divB_rel": r_div,
            "state_finite": finite,
            "clocks": clocks,
        }
        if fp32 is not None:
            line["fp32_bulk"] = fp32
        if extra is not None:
            line["order3_196608"] = extra
        if not a.no_cpu_baseline:
            try:
                line["cpu_baseline"] = cpu_baseline(a)
            except Exception as ex:  # reported, never fatal
                line["cpu_baseline"] = {"error": str(ex)[:300]}
        print(json.dumps(line), flush=True)
    mesh.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def adjoint_arm(a):
    """Differentiation workload: J = sum over the outer radial faces of phi^2 / A
    after K steps of fixed dt; the gradient wrt the initial U and phi by the
    hand-written adjoint with one checkpoint per step.  Times the forward window
    (with its checkpoint copies) and the reverse sweep with CUDA events, and
    compares <grad, d> with central differences of J along seeded directions
    (U per-variable scaled with B left out, phi the discrete curl of random edge
    values, so divergence-free).  FP64 form; with --fp32-only the forward steps run
    in the FP32-bulk form, the reverse sweep on an FP64 twin mesh, and the gradient
    is also compared with the FP64 form's."""
    import numpy as np
    import torch
    from paper_1905_02504_gb300 import autodiff, geomhd
    from paper_1905_02504_gb300.inputs import make_problem
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    prec = geomhd.GEO_FP32_BULK if a.fp32_only else geomhd.GEO_FP64
    mesh = geomhd.Mesh(a.n, a.nr, 1.0, 2.0, a.order, prec=prec)
    if a.predictor is not None:
        geomhd.geo_set_predictor(mesh.h, a.predictor)
    U0, phi0 = mesh.initial_state(make_problem(a.problem, noise=a.noise), nq_zone=a.nq_zone or None,
                                  nq_edge=a.nq_edge)
    mesh.upload(U0, phi0)
    dt = mesh.cfl_dt(a.cfl)
    Z, F, E = mesh.Z, mesh.F, mesh.E
    ref64 = geomhd.Mesh(a.n, a.nr, 1.0, 2.0, a.order) if a.fp32_only else None
    if ref64 is not None and a.predictor is not None:
        geomhd.geo_set_predictor(ref64.h, a.predictor)
    Ut0 = torch.from_numpy(np.ascontiguousarray(U0)).cuda()
    pt0 = torch.from_numpy(phi0.copy()).cuda()
    rng = np.random.default_rng(1905)
    scale = np.abs(U0).mean(axis=1)
    dirs = []
    for _ in range(a.fd_directions):
        dU = rng.uniform(-1.0, 1.0, U0.shape) * scale[:, None]
        dU[5:8] = 0.0
        dphi = geomhd.geo_phi_from_edge_circulation(mesh.h, rng.uniform(-1.0, 1.0, E) * 1e-2)
        dirs.append((torch.from_numpy(dU).cuda(), torch.from_numpy(dphi).cuda()))

    def J_of(Ux, px, K):
        geomhd.geo_state_upload(mesh.h, Ux, px)
        for _ in range(K):
            geomhd.geo_step(mesh.h, dt)
        out_U = torch.empty_like(Ux)
        out_p = torch.empty_like(px)
        geomhd.geo_state_download(mesh.h, out_U, out_p)
        return geomhd.geo_outer_Br2(mesh.h, out_p)

    results = []
    for K in [int(k) for k in a.adjoint.split(",") if k]:
        # warm-up window, then one timed forward + backward
        for timed in (False, True):
            Ut = Ut0.clone().requires_grad_(True)
            pt = pt0.clone().requires_grad_(True)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            torch.cuda.synchronize()
            e0.record()
            UK, pK = autodiff.step_window(mesh, Ut, pt, dt, K)
            J = autodiff.outer_br2(mesh, pK)
            e1.record()
            J.backward()
            e2.record()
            torch.cuda.synchronize()
        fwd_ms, bwd_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)
        gU, gphi = Ut.grad, pt.grad
        vs64 = None
        if ref64 is not None:
            # the FP64 form's gradient of the same window, for the FP32-bulk one
            U6 = Ut0.clone().requires_grad_(True)
            p6 = pt0.clone().requires_grad_(True)
            _, pK6 = autodiff.step_window(ref64, U6, p6, dt, K)
            autodiff.outer_br2(ref64, pK6).backward()
            rel = []
            for dU, dphi in dirs:
                a32 = float((gU * dU).sum() + (gphi * dphi).sum())
                a64 = float((U6.grad * dU).sum() + (p6.grad * dphi).sum())
                rel.append(abs(a32 - a64) / max(abs(a64), 1e-300))
            vs64 = {"median": float(np.median(rel)), "max": float(np.max(rel))}
        fd_stats = []
        for eps in [float(e) for e in a.fd_eps.split(",") if e]:
            errs = []
            for dU, dphi in dirs:
                adj = float((gU * dU).sum() + (gphi * dphi).sum())
                fd = (J_of(Ut0 + eps * dU, pt0 + eps * dphi, K) - J_of(Ut0 - eps * dU, pt0 - eps * dphi, K)) / (2 * eps)
                errs.append(abs(adj - fd) / max(abs(fd), 1e-300))
            errs = np.array(errs)
            fd_stats.append({"eps": eps, "directions": len(errs), "median": float(np.median(errs)),
                             "p90": float(np.quantile(errs, 0.9)), "max": float(errs.max()),
                             "within_1e-6": int((errs <= 1e-6).sum()), "within_1e-4": int((errs <= 1e-4).sum())})
        results.append({"K": K, "J": float(J.detach()), "forward_ms": fwd_ms, "backward_ms": bwd_ms,
                        "gradient_zone_updates_per_s": Z * K / ((fwd_ms + bwd_ms) * 1e-3),
                        "adjoint_over_forward": bwd_ms / fwd_ms,
                        "checkpoint_bytes": K * (8 * Z + F) * 8,
                        "fd_rel_err": fd_stats, "fp32_bulk_vs_fp64_gradient": vs64})
    if rank == 0:
        last = results[-1]
        line = {"metric": "zone-updates/s of the gradient (K forward steps with checkpoints + K adjoint steps)",
                "value": last["gradient_zone_updates_per_s"], "unit": "zone-updates/s", "n_gpus": ws,
                "steps": last["K"], "warmup": 1, "ms_per_step": (last["forward_ms"] + last["backward_ms"]) / last["K"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32-bulk forward, f64 adjoint" if a.fp32_only else "f64",
                "data": "synthetic",
                "config": {"workload": "differentiation: " + workload_name(a) + ", J = outer-shell B_r^2",
                           "zones": Z, "dt": dt},
                "windows": results}
        print(json.dumps(line), flush=True)
    mesh.close()
    if ref64 is not None:
        ref64.close()


def convergence_arm(a):
    """Design-order study of the GPU path (FP64 form unless --fp32-only): the
    entropy wave rho = 1 + 0.1 sin(2 pi (x+y+z)/sqrt3) advected by v = (0.5, 0.5,
    0.5) at uniform p and B, which the MHD equations carry exactly.  L1 error of the
    zone-averaged density at t_end over the zones whose centroid radius lies in the
    band (away from the continuative radial boundaries), against the exact zone
    averages (Gauss cubature, p + 2 points per direction); observed order
    log2(e_n / e_2n)."""
    import numpy as np
    import torch
    from paper_1905_02504_gb300 import geomhd
    from paper_1905_02504_gb300.inputs import make_problem
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    T_end = a.t_end
    r_lo, r_hi = [float(x) for x in a.shell.split(",")]
    v0 = np.array([0.5, 0.5, 0.5])
    pr = make_problem("entropy", v0=tuple(v0), B0=(0.2, 0.1, -0.1))
    prec = geomhd.GEO_FP32_BULK if a.fp32_only else geomhd.GEO_FP64
    out = {}
    for p in [int(x) for x in a.orders.split(",") if x]:
        rows = []
        for n in [int(x) for x in a.convergence.split(",") if x]:
            mesh = geomhd.Mesh(n, n, 1.0, 2.0, p, prec=prec)
            if a.predictor is not None:
                geomhd.geo_set_predictor(mesh.h, a.predictor)
            U0, phi0 = mesh.initial_state(pr)
            mesh.upload(U0, phi0)
            nst = int(np.ceil(T_end / mesh.cfl_dt(a.cfl)))
            dt = T_end / nst
            t0 = time.perf_counter()
            for _ in range(nst):
                mesh.step(dt)
            U, phi = mesh.download()
            wall = time.perf_counter() - t0
            pts, w = geomhd.geo_zone_cubature(mesh.h, p + 2)
            ex = np.einsum("zg,zg->z", w, pr.primitive(pts - T_end * v0)[0]) / w.sum(1)
            xc, vol = geomhd.geo_zone_geometry(mesh.h)
            r = np.linalg.norm(xc, axis=1)
            mask = (r > r_lo) & (r < r_hi)
            err = float(np.sum(np.abs(U[0] - ex)[mask] * vol[mask]) / np.sum(vol[mask]))
            _, rdiv = mesh.divB()
            rows.append({"n": n, "zones": mesh.Z, "steps": nst, "L1_rho": err, "divB_rel": rdiv,
                         "wall_s": wall})
            mesh.close()
            del pts, w
        for i in range(1, len(rows)):
            rows[i]["order"] = float(np.log2(rows[i - 1]["L1_rho"] / rows[i]["L1_rho"]))
        out[str(p)] = rows
    if rank == 0:
        print(json.dumps({"study": "design order, exact entropy wave, t = %g, r in (%g, %g)" % (T_end, r_lo, r_hi),
                          "form": "f32-bulk" if a.fp32_only else "f64", "cfl": a.cfl, "orders": out}),
              flush=True)


def contraction_arm(a):
    """The predictor's contraction sum_alpha D^alpha F^alpha (Eq. C.34) timed alone,
    as many times per zone as the FP32-bulk predictor performs it (level 1, then
    p Picard iterations over levels 2..M), in the CUDA-core form of the variable
    team and in a tensor-core form (mma.sync TF32, three passes), beside the
    predictor kernel's own time per step on the same mesh."""
    import numpy as np
    import torch
    from paper_1905_02504_gb300 import geomhd
    from paper_1905_02504_gb300.inputs import domain, make_problem
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    p = a.order
    a.fp32_only = True
    mesh = geomhd.Mesh(a.n, a.nr, *domain(a.problem), p, prec=geomhd.GEO_FP32_BULK, stream=stream.cuda_stream,
                       gamma=make_problem(a.problem).gamma)
    pred = default_schedule(p, True) if a.predictor is None else a.predictor
    geomhd.geo_set_predictor(mesh.h, pred)
    U0, phi0 = mesh.initial_state(make_problem(a.problem))
    mesh.upload(U0, phi0)
    dt = mesh.cfl_dt(a.cfl)
    with torch.cuda.stream(stream):
        for _ in range(a.warmup):
            mesh.step(dt)
    torch.cuda.synchronize()
    geomhd.geo_set_stage_timing(mesh.h, 1)
    with torch.cuda.stream(stream):
        for _ in range(a.steps):
            mesh.step(dt)
    torch.cuda.synchronize()
    geomhd.geo_set_stage_timing(mesh.h, 0)
    stage_ms, stage_cnt = geomhd.geo_get_stage_timing(mesh.h)
    pred_ms = stage_ms[2] / max(int(stage_cnt[2]), 1)
    Z = mesh.Z
    N = {2: 8, 3: 20, 4: 32}[p]
    nnz = {2: 16, 3: 96, 4: 192}[p]
    reps = 1 + p * (p - 1)
    out = torch.empty((Z, 8, N), dtype=torch.float32, device="cuda")
    forms = {}
    for tensor, name in ((0, "cuda_core_sparse"), (1, "mma_sync_tf32x3_dense")):
        ms = [geomhd.geo_probe_contraction(mesh.h, tensor, Z, reps, out) for _ in range(3)]
        t = float(np.median(ms))
        useful = 2.0 * 3 * nnz * 8 * reps * Z
        forms[name] = {"ms": round(t, 4), "share_of_predictor": round(t / pred_ms, 3),
                       "useful_tflops": round(useful / (t * 1e-3) / 1e12, 2)}
    mp, kp = (N + 15) // 16 * 16, (3 * N + 7) // 8 * 8
    forms["mma_sync_tf32x3_dense"]["issued_tflops"] = round(
        3 * 2.0 * mp * kp * 8 * reps * Z / (forms["mma_sync_tf32x3_dense"]["ms"] * 1e-3) / 1e12, 1)
    print(json.dumps({"study": "predictor contraction alone, FP32", "workload": workload_name(a), "order": p,
                      "zones": Z, "contractions_per_zone": reps, "predictor_schedule": sched_name(pred, p, True),
                      "predictor_ms_per_step": round(pred_ms, 4), "forms": forms}), flush=True)
    mesh.close()


def prism_arm(a):
    """The predictor on the paper's prism zones, alone: seeded synthetic frustums
    (each zone the reference prism under its own random affine map, scaled to a
    zone of a 1-2 radius shell), a smooth state with 1 % seeded noise at the
    nodes, FP64.  Inputs and outputs (several GB) exceed L2; CUDA events on the
    launching stream around each launch, after 3 warm-up launches."""
    import numpy as np
    import torch
    from paper_1905_02504_gb300 import geomhd
    torch.cuda.set_device(0)
    p, Z = a.order, a.prism_zones
    xi = geomhd.geo_prism_nodes(p)                               # (N, 3)
    N = len(xi)
    rng = np.random.default_rng(1905)
    cen = rng.normal(size=(Z, 3))
    cen *= (1.0 + rng.uniform(size=(Z, 1))) / np.linalg.norm(cen, axis=1, keepdims=True)
    A = 0.02 * (np.eye(3)[None] + 0.1 * rng.standard_normal((Z, 3, 3)))
    X = cen[:, None, :] + np.einsum("zde,ne->znd", A, xi)         # (Z, N, 3)
    g = 5.0 / 3.0
    U = np.empty((Z, N, 8))
    U[..., 0] = 1.0 + 0.01 * rng.uniform(-1.0, 1.0, (Z, N))
    U[..., 1:4] = U[..., :1] * np.array([0.3, -0.2, 0.1])
    U[..., 5:8] = np.array([0.4, -0.3, 0.2])
    U[..., 4] = 0.8 / (g - 1) + 0.5 * (U[..., 1:4] ** 2).sum(-1) / U[..., 0] + 0.5 * (U[..., 5:8] ** 2).sum(-1)
    Xd = torch.from_numpy(np.ascontiguousarray(X.transpose(2, 1, 0))).cuda()
    Ud = torch.from_numpy(np.ascontiguousarray(U.transpose(2, 1, 0))).cuda()
    del X, U
    Uh = torch.empty((p, 8, N, Z), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(3):
            geomhd.geo_prism_predictor(p, Xd, Ud, 1e-3, g, Uh, stream.cuda_stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
        for e0, e1 in ev:
            e0.record(stream)
            geomhd.geo_prism_predictor(p, Xd, Ud, 1e-3, g, Uh, stream.cuda_stream)
            e1.record(stream)
    torch.cuda.synchronize()
    ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    t = float(np.median(ms))
    ok = bool(torch.isfinite(Uh).all().item())
    print(json.dumps({"study": "ADER-CG predictor on the paper's prism zones (geo_prism_predictor), FP64",
                      "order": p, "nodes_per_zone": N, "zones": Z, "launches": a.steps, "ms_median": round(t, 4),
                      "ms_min": round(min(ms), 4), "zones_per_s": Z / (t * 1e-3), "finite": ok,
                      "inputs": "seeded affine prisms in a 1-2 shell, smooth state with 1 % noise; "
                                "inputs and outputs larger than L2"}), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        reference_arm(a)
    elif a.prism:
        prism_arm(a)
    elif a.contraction:
        contraction_arm(a)
    elif a.convergence:
        convergence_arm(a)
    elif a.adjoint:
        adjoint_arm(a)
    else:
        gpu_arm(a)


if __name__ == "__main__":
    main()
