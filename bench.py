#!/usr/bin/env python
"""Jacobian-apply throughput of the matrix-free Q_k nonlinear Stokes operator on GB300.

One step = a batch of B Newton-Jacobian applies (the hot path: gather with
R_i and the basal projector, sum-factorised gradients, pointwise Glen /
Newton physics, transposed contractions, scatter-add, basal Robin face term,
constraint rows) on B distinct seeded direction vectors resident in HBM,
using the linearised per-quadrature-point state in FP32 (the apply run inside
the Krylov iterations).  value = MDoF/s = (3 Nv + Np) * applies / time,
summed over ranks (independent replicas: the operator has no data-path
collective on one mesh per GPU).

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the CPU oracle timings (cpu_baseline, --impl reference) run on one core:
# no threaded BLAS under numpy (set before numpy is first imported)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

METRIC = "Jacobian-apply MDoF/s & %HBM roofline; time-to-1e-10 residual FP32-inner vs FP64"
UNIT = "MDoF/s"
STATE_FIELDS = 11


# Sources that define the stored-state apply kernels: a capture's DRAM
# traffic is reported only while their hash equals the one recorded with it.
KERNEL_SOURCES = [
    "paper_1406_6573_gb300/csrc/" + f for f in
    ("kernels.h", "hanging.h", "tma.cuh", "elem_kernels.cuh", "elem_body.cuh", "cpl_apply.cuh",
     "k2.cu", "k3.cu", "k4.cu")]


def kernel_source_sha():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(kernel, workload):
    """DRAM bytes (read + write) per launch of `kernel` on `workload` from the
    ncu summaries under profiles/ (a line 'traffic-record: {json}' written
    with the capture), or (None, reason) if no capture of the current kernel
    source exists."""
    sha = kernel_source_sha()
    pdir = os.path.join(ROOT, "profiles")
    stale = None
    for name in sorted(os.listdir(pdir)) if os.path.isdir(pdir) else []:
        if not name.endswith(".md"):
            continue
        for line in open(os.path.join(pdir, name)):
            if not line.startswith("traffic-record:"):
                continue
            try:
                rec = json.loads(line.split(":", 1)[1])
            except ValueError:
                continue
            if rec.get("kernel") == kernel and rec.get("workload") == workload:
                if rec.get("source_sha") == sha:
                    return int(rec["dram_bytes_per_launch"]), f"profiles/{name}"
                stale = f"profiles/{name} (kernel source changed since that capture)"
    return None, stale or "no capture of this kernel and workload"


def state_stride(k):
    """Values per element of the linearised state (the library's layout: 2
    constants, a one-value shift slot, 11 fields per quadrature point, padded
    to 16 bytes; for two elements per warp (k = 3) the stride is 16 mod 32)."""
    n1 = k + 1
    s = (2 + STATE_FIELDS * n1 ** 3 + 1 + 3) // 4 * 4
    if 32 // (n1 * n1) == 2:
        while s % 32 != 16:
            s += 4
    return s


def workload_label(wl):
    """The workload named by what it is (mesh, discretisation, size)."""
    sp = f"P{wl.k - 1}" if wl.pspace == "P" else f"Q{wl.k - 2}"
    text = (f"{wl.name}: {wl.nx}x{wl.ny}x{wl.nz} hexahedra, Q{wl.k} x {sp}^disc, "
            f"{wl.Lx / 1e3:g} km x {wl.Ly / 1e3:g} km slab")
    if wl.refine_frac == 0.0 and wl.periodic:
        npr = wl.k * (wl.k + 1) * (wl.k + 2) // 6 if wl.pspace == "P" else (wl.k - 1) ** 3
        nv = (wl.nx * wl.k) * (wl.ny * wl.k) * (wl.nz * wl.k + 1)
        text += f", {3 * nv + wl.n_coarse * npr} dofs"
    else:
        text += f", {round(100 * wl.refine_frac)} % of cells refined once"
    return text


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="slab_128x128x8_q2p1")
    ap.add_argument("--batch", type=int, default=16, help="applies per step (distinct inputs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-solve", action="store_true",
                    help="skip the time-to-1e-10 Newton solves (FP32-inner vs FP64)")
    ap.add_argument("--pairing-study", action="store_true",
                    help="Q2 x P1 against Q2 x Q0 pressure (Section 3.2.2): FP32-inner Newton solves to 1e-10 on "
                         "16 x 16 x 4 slabs of element aspect ratio phi = 1 .. 100, Krylov iterations and time")
    ap.add_argument("--adjoint-check", type=int, default=0, metavar="N",
                    help="adjoint gradient of a surface misfit and N central-difference directional checks")
    ap.add_argument("--restart", type=int, default=30, help="FGMRES restart length of the solves")
    ap.add_argument("--no-solve-profile", action="store_true",
                    help="skip the traced FP32-inner solve (device time per kernel class)")
    ap.add_argument("--velocity-mg", type=int, default=1, choices=[0, 1],
                    help="velocity block of the solver's preconditioner: 1 the column-preserving "
                         "multigrid (conforming Q2 meshes), 0 the column blocks alone")
    ap.add_argument("--eta-max", type=float, default=1e-4,
                    help="cap of the Eisenstat-Walker forcing term of the time-to-solution runs "
                         "(1e-4: with the multigrid velocity block the Krylov iterations are cheap and "
                         "fewer Newton steps pay; 128x128x8 FP32-inner 0.46 s at 0.1, 0.19 s at 1e-4)")
    ap.add_argument("--solve-precs", default="fp32_inner,fp64",
                    help="which time-to-1e-10 solves to run (comma list of fp32_inner, fp64, "
                         "fp32_inner_picard: the Picard iteration for comparison)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def clocks_start(index):
    f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    try:
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_Q}", "--format=csv,noheader,nounits",
                              "-i", str(index), "-lms", "20"], stdout=f, stderr=subprocess.DEVNULL)
    except FileNotFoundError:
        p = None
    return p, f.name


def clocks_stop(handle):
    p, path = handle
    if p is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    p.terminate()
    try:
        p.wait(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
    sm, smax, reasons, power = [], [], set(), []
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1])); smax.append(float(parts[2]))
            power.append(float(parts[3]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    os.unlink(path)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "samples": len(sm),
            "power_w_max": max(power) if power else None,
            "reasons": sorted(reasons)}


# ------------------------------------------------------------- CPU oracle
def oracle_sample(wl, n_side=8):
    """The same workload restricted to an n_side x n_side column block (same element shapes)."""
    import dataclasses
    sx = min(n_side, wl.nx)
    sy = min(n_side, wl.ny)
    return dataclasses.replace(wl, name=f"{wl.name}[{sx}x{sy}x{wl.nz} block]", nx=sx, ny=sy,
                               Lx=wl.Lx * sx / wl.nx, Ly=wl.Ly * sy / wl.ny, periodic=False,
                               refine_frac=wl.refine_frac)


def cpu_oracle_rate(wl, seconds=12.0, n_side=8, reps=None):
    """Oracle FP64 Jacobian applies on a bounded sample; returns (MDoF/s, sample text, applies)."""
    import numpy as np
    import stokes_synth as synth
    from oracle import OracleMesh, stokes as ostokes
    sw = oracle_sample(wl, n_side)
    om = OracleMesh(sw)
    lb = np.zeros(om.Nb) if sw.phys.logbeta is None else sw.phys.logbeta(*om.basal_coords()[:, :2].T)
    up = synth.uniform_vector(1, om.ndof)
    x = synth.uniform_vector(1, om.ndof, stream=1)
    ostokes.jacobian_apply(om, sw.phys, up, x, lb)   # warm
    n, t0 = 0, time.perf_counter()
    while True:
        ostokes.jacobian_apply(om, sw.phys, up, x, lb)
        n += 1
        dt = time.perf_counter() - t0
        if (reps is not None and n >= reps) or (reps is None and dt >= seconds):
            break
    rate = om.ndof * n / dt / 1e6
    text = (f"{sw.nx}x{sw.ny}x{sw.nz} column block of {wl.name} ({om.E} elements, {om.ndof} dofs), "
            f"{n} FP64 oracle Jacobian applies in {dt:.1f} s, numpy single thread")
    return rate, text, n, dt


def adjoint_check(args, wl, mesh, rank):
    """Gradient of J = 1/2 sum_top |u - u_obs|^2 with respect to log(beta) and A
    by one adjoint solve (FP32-inner solver), checked against central
    differences of forward Newton solves along seeded smooth directions.
    u_obs comes from a forward solve at a perturbed log(beta)."""
    import numpy as np
    import torch
    import stokes_synth as synth
    from paper_1406_6573_gb300 import capi
    from paper_1406_6573_gb300.adjoint import StokesForward, StokesProblem, misfit, top_nodes

    xyz = mesh.node_coords()
    bxy = xyz[mesh.basal_nodes(), :2]
    lb_ref = torch.as_tensor(wl.phys.logbeta(bxy[:, 0], bxy[:, 1]), dtype=torch.float64, device="cuda")
    prob = StokesProblem(mesh, wl.phys, inner_prec=capi.STOKES_F32, rtol=1e-11, adjoint_rtol=1e-11,
                         max_krylov=20000, max_newton=80)
    top = top_nodes(mesh)
    A = torch.tensor(wl.phys.A, dtype=torch.float64, device="cuda")

    def smooth(seed):   # a few random Fourier modes of the periodic basal plane
        rng = np.random.default_rng([seed, 77])
        f = np.zeros(len(bxy))
        for _ in range(4):
            kx, ky = rng.integers(1, 4, size=2)
            ph = rng.uniform(0, 2 * np.pi)
            f += rng.uniform(-1, 1) * np.cos(2 * np.pi * (kx * bxy[:, 0] / wl.Lx + ky * bxy[:, 1] / wl.Ly) + ph)
        return torch.as_tensor(f, device="cuda")

    with torch.no_grad():
        u_obs = StokesForward.apply(lb_ref + 0.3 * smooth(1), A, prob)[: 3 * mesh.Nv].view(-1, 3)[top].clone()
    # one untimed forward and adjoint pass: the first launches of torch's own
    # kernels on the misfit path (measured: seconds on a fresh box) stay out of
    # the timing
    lw = lb_ref.clone().requires_grad_(True)
    misfit(StokesForward.apply(lw, A, prob), u_obs, mesh, top).backward()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lb = lb_ref.clone().requires_grad_(True)
    J = misfit(StokesForward.apply(lb, A, prob), u_obs, mesh, top)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    J.backward()
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0 - t_fwd
    g = lb.grad.detach()
    h = 1e-4
    checks = []
    for d_i in range(args.adjoint_check):
        d = smooth(100 + d_i)
        with torch.no_grad():
            jp = misfit(StokesForward.apply(lb_ref + h * d, A, prob), u_obs, mesh, top).item()
            jm = misfit(StokesForward.apply(lb_ref - h * d, A, prob), u_obs, mesh, top).item()
        fd = (jp - jm) / (2 * h)
        ad = float((g * d).sum())
        checks.append(abs(fd - ad) / abs(ad))
    prob.close()
    return {"misfit": float(J), "forward_solve_s": round(t_fwd, 3), "adjoint_s": round(t_adj, 3),
            "grad_norm": float(g.norm()), "directions": args.adjoint_check, "h": h,
            "fd_rel_diff_max": max(checks), "fd_rel_diff": [float("%.3g" % c) for c in checks],
            "forward_rtol": 1e-11, "adjoint_rtol": 1e-11}


def pairing_study(args):
    """Time to 1e-10 of both pressure pairings on thin slabs of growing element
    aspect ratio phi = (L / nx) / (H / nz): the P_(k-1) pairing loses inf-sup
    stability as phi grows, the Q_(k-2) pairing does not (Section 3.2.2)."""
    import dataclasses
    import math
    import torch
    import stokes_synth as synth
    from stokes_synth.fields import bed_field, surface_field
    from paper_1406_6573_gb300 import capi
    from paper_1406_6573_gb300.mesh import Mesh, params
    out = []
    nx, nz, H = 16, 4, 1000.0
    for phi in (1.0, 4.0, 16.0, 100.0):
        L = phi * (H / nz) * nx
        for ps in ("P", "Q"):
            base = synth.workload("slab_8x8x2_q2p1")
            wl = dataclasses.replace(base, name=f"phi{phi:g}_{ps}", nx=nx, ny=nx, nz=nz, pspace=ps, Lx=L, Ly=L,
                                     bed=bed_field(base.seed, L, L, max_dev=0.05 * H),
                                     surface=surface_field(base.seed, L, L, mean=H, max_dev=0.02 * H))
            m = Mesh(wl, device=0)
            xyz = m.node_coords()
            bn = m.basal_nodes()
            lb = torch.as_tensor(wl.phys.logbeta(xyz[bn, 0], xyz[bn, 1]), dtype=torch.float64, device="cuda")
            p = params(wl.phys, lb)
            row = {"phi": phi, "pressure": "P1" if ps == "P" else "Q0", "dofs": m.ndof}
            for mg in (1, 0):
                op = capi.stokes_solver_opts()
                op.inner_prec = capi.STOKES_F32
                op.restart = 30
                op.max_krylov = 6000
                op.max_newton = 60
                op.rtol = 1e-10
                op.eta_max = args.eta_max
                op.velocity_mg = mg
                sv = capi.stokes_solver_create(m.handle, op)
                up = torch.zeros(m.ndof, dtype=torch.float64, device="cuda")
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc, rep = capi.stokes_newton_solve(sv, p, up, check=False)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                capi.stokes_solver_destroy(sv)
                key = "multigrid" if mg else "column_blocks"
                row[key] = {"converged": bool(rep["converged"]), "seconds": round(dt, 3),
                            "newton_its": rep["newton_its"], "krylov_its": rep["krylov_its"]}
            out.append(row)
            m.close()
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import stokes_synth as synth
    from oracle import OracleMesh, stokes as ostokes
    wl = synth.workload(args.workload)
    sw = oracle_sample(wl, 4)
    om = OracleMesh(sw)
    lb = np.zeros(om.Nb) if sw.phys.logbeta is None else sw.phys.logbeta(*om.basal_coords()[:, :2].T)
    up = synth.uniform_vector(1, om.ndof)
    x = synth.uniform_vector(1, om.ndof, stream=1)
    for _ in range(args.warmup):
        ostokes.jacobian_apply(om, sw.phys, up, x, lb)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ostokes.jacobian_apply(om, sw.phys, up, x, lb)
    dt = time.perf_counter() - t0
    value = om.ndof * args.steps / dt / 1e6
    sample = (f"{sw.nx}x{sw.ny}x{sw.nz} column block of {wl.name} ({om.E} elements, {om.ndof} dofs); "
              f"one FP64 oracle Jacobian apply per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded thin periodic ice slab)",
        "config": {"workload": workload_label(wl),
                   "apply": "Newton Jacobian action, FP64 oracle (dense basis tables, assembled over elements)",
                   "sample": sample, "parallelism": "host, 1 core"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------- ours
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import stokes_synth as synth
    from paper_1406_6573_gb300 import capi
    from paper_1406_6573_gb300.mesh import Mesh, State, params
    from paper_1406_6573_gb300.replicas import job_rate, max_over_ranks

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    wl = synth.workload(args.workload)
    t_build = time.perf_counter()
    mesh = Mesh(wl, device=local)
    t_build = time.perf_counter() - t_build
    ndof = mesh.ndof
    q3 = (wl.k + 1) ** 3
    n3 = (wl.k + 1) ** 3
    coords = mesh.node_coords()
    bnodes = mesh.basal_nodes()
    lb_host = (np.zeros(mesh.Nb) if wl.phys.logbeta is None
               else wl.phys.logbeta(coords[bnodes, 0], coords[bnodes, 1]))
    lb = torch.as_tensor(lb_host, dtype=torch.float64, device="cuda")
    p = params(wl.phys, lb)
    stream = torch.cuda.current_stream()

    # linearisation point: a seeded smooth-in-scale state (velocity m/a, pressure Pa)
    up = torch.as_tensor(synth.uniform_vector(rank, ndof), dtype=torch.float64, device="cuda")
    up[: 3 * mesh.Nv] *= 100.0
    up[3 * mesh.Nv:] *= 1e5
    st = State(mesh, capi.STOKES_F32)
    st.linearize(p, up)
    B = args.batch
    gen = torch.Generator(device="cuda").manual_seed(1000 + rank)
    X = [torch.rand(ndof, dtype=torch.float32, device="cuda", generator=gen) * 2 - 1 for _ in range(B)]
    Y = [torch.empty(ndof, dtype=torch.float32, device="cuda") for _ in range(B)]

    def step():
        for b in range(B):
            st.apply(X[b], Y[b], stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ck = clocks_start(local)
    time.sleep(0.1)
    capi.stokes_profile_begin(mesh.handle)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    prof = capi.stokes_profile_end(mesh.handle)
    clocks = clocks_stop(ck)
    barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), "cuda")
    applies = args.steps * B
    value = job_rate(ndof * applies, ms / 1e3, "cuda") / 1e6

    # roofline of the dominant kernel (volume element kernel of the FP32 state apply)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    el_launches, el_ms = prof["element"]
    el_avg_s = el_ms / max(el_launches, 1) / 1e3
    sstride = state_stride(wl.k)
    # element kernel of one apply (it also does the basal Robin term and the
    # constraint rows): state, x read and y written once, basal index per
    # element, element map and hanging code where the kernel reads them (not
    # on conforming lattice meshes, whose nodes follow from the element
    # index), basal face geometry and map, log(beta), basal node list and
    # projector
    mask = wl.refine_mask().reshape(wl.nz, wl.ny, wl.nx)[0]
    refined = bool(wl.refine_mask().any())
    n_faces = int(wl.nx * wl.ny + 3 * mask.sum())
    q2 = (wl.k + 1) ** 2
    cpl = wl.k == 2 and not refined
    if cpl:
        # component-per-lane kernel: basal Robin term of the basal elements in
        # the element pass from the FP32 basal state (beta w |J_s|, n: 4 values
        # per face Gauss point; 10 with the nonlinear sliding law), the face
        # index and the FP32 projector rows of the basal elements; constraint
        # rows: basal node list and FP64 projector
        nf = 10 if getattr(wl.phys, "sliding_m", 1.0) not in (0.0, 1.0) else 4
        bytes_basal = (n_faces * (nf * q2 * 4 + 4 + 6 * q2 * 4) if wl.phys.robin else 0) + mesh.Nb * (4 + 48)
    else:
        bytes_basal = (n_faces * (4 * q2 * 8 + q2 * 4) + mesh.Nb * (8 + 4 + 48)) if wl.phys.robin else mesh.Nb * 52
    bytes_desc = mesh.E * 4 + (mesh.E * (n3 * 4 + 4) if refined else 0)
    bytes_alg = mesh.E * sstride * 4 + 2 * ndof * 4 + bytes_desc + bytes_basal
    achieved = bytes_alg / el_avg_s / 1e9
    kname = ("cpl_state_apply_kernel<%d,false>" % (0 if wl.pspace == "P" else 1)
             if (wl.k == 2 and not refined) else "state_apply_kernel<float,false>")
    traffic, traffic_src = captured_traffic(kname, wl.name)
    shares = {k: v[1] for k, v in prof.items()}
    tot = sum(shares.values())

    # e2e: host buffers, host<->device copies inside the timed region
    e2e = None
    if not args.no_e2e:
        Xh = [x.cpu().pin_memory() for x in X]
        Yh = [torch.empty(ndof, dtype=torch.float32).pin_memory() for _ in range(B)]
        Xd = [torch.empty_like(x) for x in X]
        ke = max(1, min(args.steps, 50))
        # host -> device copies on one copy stream, device -> host on another,
        # the applies on the compute stream: input b + 1 and output b - 1 move
        # while apply b runs (the link is full duplex)
        s_h2d, s_d2h = torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(B)]
        ev_out = [torch.cuda.Event() for _ in range(B)]
        def e2e_step():
            s_h2d.wait_stream(stream)          # inputs of the previous step are consumed
            for b in range(B):
                with torch.cuda.stream(s_h2d):
                    Xd[b].copy_(Xh[b], non_blocking=True)
                    ev_in[b].record(s_h2d)
            for b in range(B):
                stream.wait_event(ev_in[b])
                st.apply(Xd[b], Y[b], stream)
                ev_out[b].record(stream)
                s_d2h.wait_event(ev_out[b])
                with torch.cuda.stream(s_d2h):
                    Yh[b].copy_(Y[b], non_blocking=True)
            stream.wait_stream(s_d2h)          # outputs are on the host before the next step
        e2e_step()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(ke):
            e2e_step()
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, "cuda")
        e2e = {"value": job_rate(ndof * B * ke, dt, "cuda") / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": B * ndof * 4, "d2h_bytes_per_step": B * ndof * 4,
               "steps": ke}

    # other operators of the path, timed briefly (device time per call)
    variants = {}
    if not args.no_variants and rank == 0:
        def tm(fn, n=10):
            fn(); torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(n):
                fn()
            b.record(stream); torch.cuda.synchronize()
            return a.elapsed_time(b) / n
        x64 = X[0].double()
        y64 = torch.empty(ndof, dtype=torch.float64, device="cuda")
        st64 = State(mesh, capi.STOKES_F64)
        st64.linearize(p, up)
        up32 = up.float()
        g = torch.empty(mesh.Nb, dtype=torch.float64, device="cuda")
        gA = torch.empty(1, dtype=torch.float64, device="cuda")
        v = {
            "state_apply_f64": tm(lambda: st64.apply(x64, y64, stream)),
            "state_apply_f32": tm(lambda: st.apply(X[0], Y[0], stream)),
            "jacobian_fused_f64": tm(lambda: capi.stokes_jacobian_apply(mesh.handle, p, up, x64, y64, 0, stream), 3),
            "jacobian_fused_f32": tm(lambda: capi.stokes_jacobian_apply(mesh.handle, p, up32, X[0], Y[0], 1, stream)),
            "jacobian_transpose_f32": tm(lambda: capi.stokes_jacobian_apply_transpose(mesh.handle, p, up32, X[0], Y[0], 1, stream)),
            "residual_f64": tm(lambda: capi.stokes_residual(mesh.handle, p, up, y64, 0, stream), 3),
            "residual_f32": tm(lambda: capi.stokes_residual(mesh.handle, p, up32, Y[0], 1, stream)),
            "linearize_f64_to_f32": tm(lambda: st.linearize(p, up, stream), 3),
            "param_grad_f64": tm(lambda: capi.stokes_param_grad(mesh.handle, p, up, x64, g, gA, stream), 3),
        }
        variants = {k: {"ms": round(val, 4), "MDoF/s": round(ndof / (val / 1e3) / 1e6, 1)} for k, val in v.items()}
        del st64

    # time to a 1e-10 relative residual from u = 0: FP32-inner / FP64-outer vs plain FP64
    solve = None
    if not args.no_solve:
        solve = {}
        want = set(args.solve_precs.split(","))
        import dataclasses
        p_picard = params(dataclasses.replace(wl.phys, linearization="picard"), lb)
        for tag, inner in (("fp32_inner", capi.STOKES_F32), ("fp64", capi.STOKES_F64),
                           ("fp32_inner_picard", capi.STOKES_F32)):
            if tag not in want:
                continue
            p_solve = p_picard if tag.endswith("picard") else p
            op = capi.stokes_solver_opts()
            op.inner_prec = inner
            op.restart = args.restart
            op.max_krylov = 4000
            op.max_newton = 300 if tag.endswith("picard") else 60
            op.rtol = 1e-10
            op.eta_max = args.eta_max
            op.velocity_mg = args.velocity_mg
            sv = capi.stokes_solver_create(mesh.handle, op)
            u0 = torch.zeros(ndof, dtype=torch.float64, device="cuda")
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, rep = capi.stokes_newton_solve(sv, p_solve, u0, stream, check=False)
            torch.cuda.synchronize()
            wall = max_over_ranks(time.perf_counter() - t0, "cuda")
            capi.stokes_solver_destroy(sv)
            solve[tag] = {"seconds": round(wall, 4), "converged": rep["converged"],
                          "newton_its": rep["newton_its"], "krylov_its": rep["krylov_its"],
                          "mg_levels": rep["mg_levels"],
                          "final_rel_residual": rep["res_final"] / rep["res0"]}
            if tag == "fp32_inner":
                u_fp32 = u0
            elif "fp32_inner" in solve:
                du = (u0 - u_fp32).norm() / u0.norm()
                solve["rel_diff_fp32_vs_fp64_solution"] = float(du)
        solve["eta_max"] = args.eta_max
        solve["restart"] = args.restart
        if "fp32_inner" in want and not args.no_solve_profile:
            # one more FP32-inner solve with the library's event tracing on:
            # device time per class against the wall time of that solve
            op = capi.stokes_solver_opts()
            op.inner_prec = capi.STOKES_F32
            op.restart = args.restart
            op.max_krylov = 4000
            op.max_newton = 60
            op.rtol = 1e-10
            op.eta_max = args.eta_max
            op.velocity_mg = args.velocity_mg
            sv = capi.stokes_solver_create(mesh.handle, op)
            u0 = torch.zeros(ndof, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            capi.stokes_profile_begin(mesh.handle)
            t0 = time.perf_counter()
            rc, rep = capi.stokes_newton_solve(sv, p, u0, stream, check=False)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            pr = capi.stokes_profile_end(mesh.handle)
            capi.stokes_solver_destroy(sv)
            dev_ms = sum(v[1] for v in pr.values())
            solve["fp32_inner_traced"] = {
                "seconds": round(wall, 4), "krylov_its": rep["krylov_its"],
                "device_ms": {k: [v[0], round(v[1], 2)] for k, v in pr.items() if v[0]},
                "device_ms_total": round(dev_ms, 2),
                "not_in_kernels_ms": round(wall * 1e3 - dev_ms, 2)}
        if "fp32_inner" in solve and "fp64" in solve:
            solve["speedup_fp32_inner"] = round(solve["fp64"]["seconds"] / solve["fp32_inner"]["seconds"], 3)

    adjoint = adjoint_check(args, wl, mesh, rank) if args.adjoint_check > 0 else None
    pairing = pairing_study(args) if args.pairing_study and rank == 0 else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, text, n, dt = cpu_oracle_rate(wl, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": text}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded thin periodic ice slab, random-Fourier bed and surface)",
            "config": {
                "workload": workload_label(wl),
                "apply": "Newton Jacobian from the stored FP32 linearised state (Krylov-inner apply)",
                "applies_per_step": B,
                "l2": "inputs larger than L2 (FP32 state %d MB + %d distinct x/y pairs of %d MB)"
                      % (mesh.E * sstride * 4 // 2**20, B, ndof * 4 // 2**20),
                "parallelism": f"replicas{world}",
                "mesh_build_s": round(t_build, 2),
            },
            "clocks": clocks,
            "gpu_launches": int(prof["element"][0] + prof["face"][0] + prof["constraint"][0]),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak,
                         "traffic": traffic,
                         "traffic_source": traffic_src,
                         "kernel": kname,
                         "bytes_per_launch": bytes_alg, "avg_launch_ms": el_avg_s * 1e3,
                         "peak_source": f"{peak_src} hbm_gbs"},
            "kernel_time_share": {k: round(v / tot, 4) for k, v in shares.items()} if tot > 0 else {},
            "e2e": e2e,
            "time_to_1e-10": solve,
            "variants": variants,
            "cpu_baseline": cpu,
            "adjoint_check": adjoint,
        }
        if pairing is not None:
            out["pairing_study"] = pairing
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
