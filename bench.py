"""Benchmark: HMC trajectories/s of the honeycomb-Hubbard hot path on GB300.

One step = one HMC trajectory (heat bath, chi = M rho, n_md + 1 CG solves
with forces, leapfrog, Metropolis) of the chosen workload, run by
hmc_trajectory as one persistent launch.  Default workload: the largest
single-GPU configuration, L=24 (1152 sites), Nt=96, U=4, beta=12, 30
leapfrog steps over tau=1, mixed precision (FP16-split tensor-core
contraction, FP32 CG with FP64 reliable updates), thermalised from a cold
start by untimed trajectories.  The same line carries the plain FP64 GPU
path on the same field and pseudofermion source (per solve, scaled to a
trajectory), M-applications/s with their tensor-core and HBM roofline
fractions, and the oracle on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--precision fp64|mixed] [--impl ours|reference]

N > 1 (torchrun): each rank advances its own chain (chain id = rank): weak
scaling, no collective on the data path.  Prints one JSON line on rank 0.
"""
import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("HMC trajectories/s and M-applications/s (frac. of roofline), "
          "mixed vs FP64 at equal tol")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILES = os.path.join(ROOT, "profiles")
CSRC = os.path.join(ROOT, "paper_2210_06874_gb300", "csrc")
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# untimed trajectories from the cold start before the warm-up ones
THERM = {"l3_nt8": 0, "l6_nt32": 20, "l12_nt64": 10, "l24_nt96": 5}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="l24_nt96")
    ap.add_argument("--integrator", default="leapfrog", choices=["leapfrog", "omelyan"],
                    help="trajectory mode: molecular-dynamics integrator (the workload's "
                         "configuration is leapfrog)")
    ap.add_argument("--n-md", type=int, default=None,
                    help="trajectory mode: steps per trajectory (default: the workload's)")
    ap.add_argument("--precision", default=None, choices=[None, "fp64", "mixed"])
    ap.add_argument("--hb-inner", type=int, default=0,
                    help="trajectory mode, FP64: mass preconditioning with this many inner "
                         "leapfrog steps per outer step (0: off; n_md counts outer steps)")
    ap.add_argument("--hb-gamma", type=float, default=0.5,
                    help="hop factor g of the heavy operator M_g = 1 - g S E D")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="trajectory", choices=["trajectory", "apply", "brs", "cg"],
                    help="trajectory: HMC trajectories/s; apply: M-applications/s; cg: "
                         "M-applications/s inside the mixed CG (us per FP32 iteration)")
    ap.add_argument("--cg-iters", type=int, default=400,
                    help="cg mode: FP32 iterations of the longer timed solve")
    ap.add_argument("--brs-L", type=int, default=102, help="brs mode: lattice size")
    ap.add_argument("--brs-Nt", type=int, default=256, help="brs mode: time slices")
    ap.add_argument("--applies", type=int, default=20,
                    help="apply mode: applications of M per step")
    ap.add_argument("--chains", type=int, default=256, help="batch workload: chains")
    ap.add_argument("--batch-team", type=int, default=4,
                    help="batch workload: CTAs of the cluster teams that the most expensive "
                         "chains run on (1: every chain on one CTA)")
    ap.add_argument("--loop-chains", type=int, default=32,
                    help="batch workload: chains timed as a loop of single-chain launches")
    ap.add_argument("--loop-chains-fp64", type=int, default=8,
                    help="batch workload: chains timed as a loop of plain FP64 launches")
    ap.add_argument("--therm", type=int, default=None,
                    help="untimed thermalisation trajectories before warm-up")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-arm", action="store_true",
                    help="trajectory mode, mixed: skip the plain FP64 GPU path's solve")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--no-batch-line", action="store_true",
                    help="default workload: skip the batched workload's comparison that the "
                         "line carries as its batch256 object")
    ap.add_argument("--operand-mode", type=int, default=None, choices=[0, 1, 2, 3, 4, 5],
                    help="operand_mode of the mixed path instead of the autotuner's choice "
                         "(1 site-major tiles, 3 CUDA-core cluster mode, 4 slice-major "
                         "tiles, 5 split-K tiles with E resident)")
    ap.add_argument("--cpu-sample-s", type=float, default=15.0)
    return ap.parse_args()


def aggregate_rate(local_ms, units_per_rank, world, dist=None, device=None):
    """Whole-job rate of independent replicas: every rank processed
    units_per_rank units; the job took the slowest rank's time (max over
    ranks).  Returns (units per second over all ranks, max ms)."""
    ms = float(local_ms)
    if world > 1:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * units_per_rank / (ms * 1e-3), ms


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return dict(FALLBACK), "fallback"


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
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
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- helpers
def workload_params(name, precision):
    from paper_2210_06874_gb300 import hmc, synth
    w = dict(synth.WORKLOADS[name])
    prec = precision or w["precision"]
    p = hmc.Params(L=w["L"], Nt=w["Nt"], kappa=w["kappa"], U=w["U"], beta=w["beta"],
                   n_md=w["n_md"], traj_length=w["traj_length"], cg_tol=w["cg_tol"],
                   cg_max_iter=200000,
                   precision=hmc.PREC_FP64 if prec == "fp64" else hmc.PREC_MIXED)
    return w, p, prec


def flops_per_apply(V, Nt):
    """Algorithmic FLOPs of one M or M^dag application: the real V x V by
    V x 2Nt contraction (4 V^2 Nt) plus phase, shift and subtraction
    (~10 V Nt)."""
    return 4.0 * V * V * Nt + 10.0 * V * Nt



def fp32_fma_tflops(torch, dev):
    """FP32 FMA peak of the whole GPU from unit counts: SMs (device
    attribute) x 128 FP32 lanes x 2 flop x the maximum SM clock."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks, _ = load_peaks()
    mhz = peaks.get("sm_max_mhz", 2070.0)
    return sms * 128 * 2 * mhz * 1e6 / 1e12, sms, mhz


def sources_sha():
    """Hash of the library's CUDA sources (the counters of a profile are only
    valid for the kernels they were taken on)."""
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(CSRC, "*"))):
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(workload, key):
    """DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per unit
    recorded by a committed ncu summary under profiles/ for this workload, as
    a line `traffic <workload> <key> <bytes> sources <sha>`; None when there
    is none or the kernels changed since (the sha of csrc/ differs)."""
    import glob
    import re
    sha = sources_sha()
    pat = re.compile(r"^traffic\s+(\S+)\s+(\S+)\s+([0-9.eE+]+)\s+sources\s+([0-9a-f]+)")
    for f in sorted(glob.glob(os.path.join(PROFILES, "*.md"))):
        with open(f) as fh:
            for ln in fh:
                m = pat.match(ln.strip().strip("`"))
                if m and m.group(1) == workload and m.group(2) == key:
                    if m.group(4) != sha:
                        return None, "%s: kernels changed since the capture" % os.path.basename(f)
                    return float(m.group(3)), os.path.basename(f)
    return None, "no committed capture for this workload"


def flush_l2(buf, acc):
    """Evict the L2 between timed regions: a write larger than the L2, then a
    read sweep of it, so the L2 holds clean lines and the timed work pays
    no write-back of the flush's dirty lines."""
    import torch
    buf.fill_(1.0)
    torch.sum(buf, dim=0, out=acc)

def e2e_host_calls(torch, stream, dev_in, dev_out, call, n):
    """End to end through the C ABI with host buffers: n times, copy the
    input from pinned host memory to the device, call, copy the output back
    to pinned host memory; returns (ms per call, bytes in, bytes out)."""
    h_in = torch.empty(dev_in.shape, dtype=dev_in.dtype, pin_memory=True)
    h_in.copy_(dev_in.cpu())
    h_out = torch.empty(dev_out.shape, dtype=dev_out.dtype, pin_memory=True)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(n):
        dev_in.copy_(h_in, non_blocking=True)
        call()
        h_out.copy_(dev_out, non_blocking=True)
    e.record(stream)
    e.synchronize()
    nb_in = dev_in.numel() * dev_in.element_size()
    nb_out = dev_out.numel() * dev_out.element_size()
    return s.elapsed_time(e) / n, nb_in, nb_out


def applies_per_traj(out, n_md):
    """M / M^dag applications in one trajectory: chi = M rho, two per CG
    iteration, two per FP64 true-residual check (one per solve and one per
    reliable update), one M^dag per force (one force per solve, whatever the
    integrator)."""
    return 1 + 2 * out.cg_iterations + 2 * (out.cg_solves + out.reliable_updates) + out.cg_solves


def measure_dgemm_tflops(torch):
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        a @ b
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = 1e30
    for _ in range(5):
        s.record()
        a @ b
        e.record()
        e.synchronize()
        best = min(best, s.elapsed_time(e))
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def cpu_oracle_rate(name, prec, sample_s, phi_np=None, integrator="leapfrog", n_md=None,
                    hb=None):
    """Time the CPU oracle (as it stands) on trajectories of the same workload
    (and integrator; hb = (g, inner steps): mass preconditioning) until
    about sample_s seconds of work are done."""
    import numpy as np
    from oracle import hmc as ohmc, lattice, operators as ops
    from paper_2210_06874_gb300 import synth
    w = synth.WORKLOADS[name]
    delta = w["beta"] / w["Nt"]
    E = ops.transfer_matrix(lattice.hopping_matrix(w["L"]), delta * w["kappa"])
    phi = synth.start_field(name) if phi_np is None else phi_np
    t0 = time.perf_counter()
    n = 0
    iters = 0
    n_md = n_md or w["n_md"]
    while True:
        if hb:
            from oracle import hasenbusch as ohb
            out = ohb.trajectory(E, phi, delta, w["U"], hb[0], w["traj_length"] / n_md, n_md,
                                 hb[1], w["seed"], 10_000 + n, 0, tol=w["cg_tol"],
                                 max_iter=200000)
            out["cg_iters"] = out["cg_iters_inner"] + out["cg_iters_outer"]
        else:
            out = ohmc.trajectory(E, phi, delta, w["U"], w["traj_length"] / n_md, n_md,
                                  w["seed"], 10_000 + n, 0, tol=w["cg_tol"], max_iter=200000,
                                  integrator=integrator)
        phi = out["phi"]
        iters += out["cg_iters"]
        n += 1
        if time.perf_counter() - t0 > sample_s:
            break
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "trajectories/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": "%d oracle trajectories of %s (%d CG iterations), %.1f s; NumPy FP64, "
                      "BLAS threads as configured" % (n, name, iters, dt)}


def cpu_oracle_cg_iter_time(name, phi_np, chi_np, sample_s):
    """Seconds per FP64 CG iteration of the oracle (as it stands) on the
    workload's lattice: its cg_solve from x0 = 0 on (phi, chi), capped at as
    many iterations as fit in about sample_s seconds (a short first run
    sizes the cap).  Returns (seconds per iteration, iterations timed, s)."""
    from oracle import hmc as ohmc, lattice, operators as ops
    from paper_2210_06874_gb300 import synth
    w = synth.WORKLOADS[name]
    delta = w["beta"] / w["Nt"]
    E = ops.transfer_matrix(lattice.hopping_matrix(w["L"]), delta * w["kappa"])
    t0 = time.perf_counter()
    _, it0, _ = ohmc.cg_solve(E, phi_np, chi_np, tol=1e-300, max_iter=3)
    per = (time.perf_counter() - t0) / max(it0, 1)
    cap = max(3, int(sample_s / per))
    t0 = time.perf_counter()
    _, it, _ = ohmc.cg_solve(E, phi_np, chi_np, tol=1e-300, max_iter=cap)
    dt = time.perf_counter() - t0
    return dt / max(it, 1), it, dt


def cpu_oracle_rate_by_iterations(name, phi_np, chi_np, sample_s, iters_per_solve, n_solves,
                                  single_thread=False):
    """Oracle trajectories/s for workloads whose trajectory takes the oracle
    minutes: seconds per FP64 CG iteration, timed on a bounded sample, times
    the FP64 CG iterations of one trajectory (n_solves solves of
    iters_per_solve iterations from x0 = 0, the oracle's own algorithm)."""
    if single_thread:
        import tempfile
        import numpy as np
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
                   MKL_NUM_THREADS="1", BLIS_NUM_THREADS="1")
        fd, path = tempfile.mkstemp(suffix=".npz")
        os.close(fd)
        np.savez(path, phi=phi_np, chi=chi_np)
        code = ("import json, sys, numpy as np; sys.path.insert(0, %r); import bench; "
                "d = np.load(%r); print(json.dumps(bench.cpu_oracle_cg_iter_time(%r, d['phi'], "
                "d['chi'], %r)))" % (ROOT, path, name, sample_s))
        try:
            r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True,
                               text=True, timeout=sample_s * 10 + 120)
            per, it, dt = json.loads(r.stdout.strip().splitlines()[-1])
        except Exception as e:   # a reporting extra: never fail the bench on it
            return {"unavailable": str(e)[:200]}
        finally:
            os.unlink(path)
        cores, how = 1, "one thread"
    else:
        per, it, dt = cpu_oracle_cg_iter_time(name, phi_np, chi_np, sample_s)
        cores, how = os.cpu_count(), "BLAS threads as configured"
    total = iters_per_solve * n_solves
    return {"value": 1.0 / (per * total), "unit": "trajectories/s", "cores": cores,
            "kind": "oracle", "cg_iterations_per_s": 1.0 / per,
            "sample": "%d FP64 CG iterations of the oracle on %s (%.1f s, %.2f ms each), "
                      "scaled to one trajectory of %d solves x %d iterations from x0 = 0 "
                      "(the plain FP64 GPU path's count on the same field and source, "
                      "the oracle's algorithm); NumPy FP64, %s"
                      % (it, name, dt, 1e3 * per, n_solves, iters_per_solve, how)}


def cpu_oracle_rate_single_thread(name, prec, sample_s, phi_np=None, integrator="leapfrog",
                                  n_md=None):
    """The same oracle timing in a child process with BLAS and OpenMP pinned
    to one thread (thread counts are fixed when NumPy loads its BLAS); the
    start field goes through a temporary .npy file."""
    import tempfile
    import numpy as np
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1", BLIS_NUM_THREADS="1")
    fd, path = tempfile.mkstemp(suffix=".npy")
    os.close(fd)
    if phi_np is not None:
        np.save(path, phi_np)
    code = ("import json, sys, numpy as np; sys.path.insert(0, %r); import bench; "
            "phi = np.load(%r) if %r else None; "
            "print(json.dumps(bench.cpu_oracle_rate(%r, %r, %r, phi_np=phi, integrator=%r, "
            "n_md=%r)))"
            % (os.path.dirname(os.path.abspath(__file__)), path, phi_np is not None, name, prec,
               sample_s, integrator, n_md))
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True,
                           text=True, timeout=sample_s * 10 + 120)
        out = json.loads(r.stdout.strip().splitlines()[-1])
        out["cores"] = 1
        out["sample"] = out["sample"].replace("BLAS threads as configured", "one thread")
        return out
    except Exception as e:   # a reporting extra: never fail the bench on it
        return {"unavailable": str(e)[:200]}
    finally:
        os.unlink(path)


def cpu_oracle_apply_rate(name, sample_s):
    """Time the oracle's matrix-free M (as it stands) on the workload's
    lattice: applications per second over about sample_s seconds."""
    import numpy as np
    from oracle import lattice, operators as ops
    from paper_2210_06874_gb300 import synth
    w = synth.WORKLOADS[name]
    L, Nt = w["L"], w["Nt"]
    V, delta = 2 * L * L, w["beta"] / w["Nt"]
    E = ops.transfer_matrix(lattice.hopping_matrix(L), delta * w["kappa"])
    phi = synth.gaussian_field(w["seed"], Nt, V, delta * w["U"])
    psi = synth.complex_gaussian(w["seed"] + 1, Nt, V)
    t0 = time.perf_counter()
    n = 0
    while True:
        psi = ops.apply_M(E, phi, psi)
        psi /= np.linalg.norm(psi)
        n += 1
        if time.perf_counter() - t0 > sample_s:
            break
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "M-applications/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": "%d oracle applications of M on %s, %.1f s; NumPy FP64, BLAS threads "
                      "as configured" % (n, name, dt)}


def cpu_oracle_batch_rate(n_chains, sample_s, per_class=None, fields=None):
    """The oracle on the batched workload.  With per_class (the GPU arm's FP64
    sample: one chain per (L, Nt) class, its field in `fields`, its FP64 CG
    iterations per trajectory): for every class, the oracle's seconds per
    FP64 CG iteration on that chain's field and lattice (a bounded run split
    evenly over the classes), times the iterations of one of its
    trajectories, times the class's chain count; trajectories/s = chains /
    sum.  Without it: oracle trajectories of the chains in batch order from a
    cold start until about sample_s seconds of work are done."""
    import numpy as np
    from oracle import hmc as ohmc, lattice, operators as ops
    from paper_2210_06874_gb300 import synth
    specs = synth.batch256(n_chains=n_chains)
    if per_class:
        t0 = time.perf_counter()
        share = sample_s / len(per_class)
        total_s, parts = 0.0, []
        for pc in per_class:
            c = specs[pc["sampled_chain"]]
            V, delta = 2 * c["L"] ** 2, c["beta"] / c["Nt"]
            E = ops.transfer_matrix(lattice.hopping_matrix(c["L"]), delta * c["kappa"])
            phi = fields[pc["sampled_chain"]]
            rho = synth.complex_gaussian(pc["sampled_chain"] + 11, c["Nt"], V) / np.sqrt(2.0)
            chi = ops.apply_M(E, phi, rho)
            t1 = time.perf_counter()
            _, it0, _ = ohmc.cg_solve(E, phi, chi, tol=1e-300, max_iter=3)
            per = (time.perf_counter() - t1) / max(it0, 1)
            # at most a quarter of the dimension: on small lattices CG would
            # otherwise reach the exact solution and divide by a zero norm
            cap = max(3, min(int(share / per), V * c["Nt"] // 4))
            t1 = time.perf_counter()
            _, it, _ = ohmc.cg_solve(E, phi, chi, tol=1e-300, max_iter=cap)
            per = (time.perf_counter() - t1) / max(it, 1)
            total_s += per * pc["cg_iterations"] * pc["chains"]
            parts.append("L%d Nt%d: %d its x %.3f ms" % (pc["L"], pc["Nt"], pc["cg_iterations"],
                                                           1e3 * per))
        dt = time.perf_counter() - t0
        return {"value": n_chains / total_s, "unit": "trajectories/s", "cores": os.cpu_count(),
                "kind": "oracle",
                "sample": "per (L, Nt) class: oracle FP64 CG iterations timed on the sampled "
                          "chain's field after the timed steps (%.1f s in all), scaled by that "
                          "chain's FP64 CG iterations per trajectory on the GPU's FP64 path and "
                          "by the class's chain count (%d classes, %d chains; %s); NumPy FP64, "
                          "BLAS threads as configured"
                          % (dt, len(per_class), n_chains, "; ".join(parts))}
    t0 = time.perf_counter()
    n = 0
    for i, c in enumerate(specs):
        V, delta = 2 * c["L"] ** 2, c["beta"] / c["Nt"]
        E = ops.transfer_matrix(lattice.hopping_matrix(c["L"]), delta * c["kappa"])
        ohmc.trajectory(E, np.zeros((c["Nt"], V)), delta, c["U"],
                        c["traj_length"] / c["n_md"], c["n_md"], synth.BASE_SEED + 3, 0, i,
                        tol=c["cg_tol"], max_iter=200000)
        n += 1
        if time.perf_counter() - t0 > sample_s:
            break
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "trajectories/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": "oracle trajectories of the first %d of the %d chains (batch order, cold "
                      "start), %.1f s; NumPy FP64, BLAS threads as configured"
                      % (n, n_chains, dt)}


# ----------------------------------------------------------------- reference arm
def reference_iteration_setup(name, args):
    """For workloads whose oracle trajectory takes minutes to hours: the
    start field, the heat-bath source chi = M rho of its first solve, and the
    oracle's own CG iteration count for that solve (x0 = 0, the workload's
    tolerance).  The steps then time oracle CG iterations and scale them by
    that count: the first solve from the start field is the cheapest of the
    chain, so the estimate favours the oracle."""
    import math
    from oracle import hmc as ohmc, lattice, operators as ops
    from paper_2210_06874_gb300 import synth
    w = synth.WORKLOADS[name]
    delta = w["beta"] / w["Nt"]
    V = 2 * w["L"] ** 2
    E = ops.transfer_matrix(lattice.hopping_matrix(w["L"]), delta * w["kappa"])
    phi = synth.start_field(name)
    rho = synth.complex_gaussian(w["seed"] + 77, w["Nt"], V) / math.sqrt(2.0)
    chi = ops.apply_M(E, phi, rho)
    _, iters, _ = ohmc.cg_solve(E, phi, chi, tol=w["cg_tol"], max_iter=200000)
    n_md = args.n_md or w["n_md"]
    n_solves = (2 * n_md if args.integrator == "omelyan" else n_md) + 1
    return phi, chi, iters, n_solves


def run_reference(args):
    """The oracle as it stands, on the host cores, for the workload and
    metric of our arm: trajectories/s (single chain or the batched chains)
    or M-applications/s (--mode apply)."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    from paper_2210_06874_gb300 import synth
    name = args.workload
    sample_s = min(args.cpu_sample_s, 20.0)
    if args.mode == "brs":
        print(json.dumps({"impl": "reference", "unavailable":
                          "the oracle's Eq. (2.2) operator holds the dense V x V hopping "
                          "matrix: 3.5 GB and 2e11 flops per application at L = 102"}),
              flush=True)
        return
    batch = name.startswith("batch")
    apply = args.mode in ("apply", "cg") and not batch
    by_iters = None
    if not batch and not apply and 2 * synth.WORKLOADS[name]["L"] ** 2 >= 288:
        by_iters = reference_iteration_setup(name, args)
    rates, samples, secs = [], [], []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        if batch:
            r = cpu_oracle_batch_rate(args.chains, sample_s)
        elif apply and args.mode == "cg":
            w = synth.WORKLOADS[name]
            V, Nt = 2 * w["L"] ** 2, w["Nt"]
            phi0 = synth.gaussian_field(w["seed"], Nt, V, w["beta"] / Nt * w["U"], scale=0.3)
            chi0 = synth.complex_gaussian(w["seed"] + 1, Nt, V)
            per, it, dt = cpu_oracle_cg_iter_time(name, phi0, chi0, sample_s)
            r = {"value": 2.0 / per, "unit": "M-applications/s", "cores": os.cpu_count(),
                 "kind": "oracle",
                 "sample": "%d FP64 CG iterations of the oracle on %s (%.1f s), two "
                           "applications each; NumPy FP64, BLAS threads as configured"
                           % (it, name, dt)}
        elif apply:
            r = cpu_oracle_apply_rate(name, sample_s)
        elif by_iters:
            phi0, chi0, iters0, n_solves = by_iters
            r = cpu_oracle_rate_by_iterations(name, phi0, chi0, sample_s, iters0, n_solves)
            r["sample"] = r["sample"].replace(
                "(the plain FP64 GPU path's count on the same field and source, the oracle's "
                "algorithm)", "(the oracle's own count for the first solve from the workload's "
                "start field, the cheapest solve of the chain)")
        else:
            r = cpu_oracle_rate(name, None, sample_s, integrator=args.integrator,
                                n_md=args.n_md)
        if k >= args.warmup:
            rates.append(r["value"])
            samples.append(r["sample"])
            secs.append(time.perf_counter() - t0)
    value = statistics.mean(rates)
    unit = "M-applications/s" if apply else "trajectories/s"
    if batch:
        config = {"workload": name, "precision": "fp64 (oracle)", "chains": args.chains}
    else:
        w = synth.WORKLOADS[name]
        config = {"workload": name, "precision": "fp64 (oracle)", "L": w["L"], "Nt": w["Nt"]}
        if apply:
            config["mode"] = args.mode
        else:
            config.update(n_md=args.n_md or w["n_md"], integrator=args.integrator)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": unit,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
        "cpu_baseline": {"value": value, "unit": unit, "cores": os.cpu_count(),
                         "kind": "oracle",
                         "sample": "each step ~%.0f s of oracle work; last step: %s"
                                   % (sample_s, samples[-1])},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- our arm
def fp64_vs_mixed_solve(ctx, params, phi, seed, dev):
    """The plain FP64 GPU path against the mixed path on one pseudofermion
    solve of the current field: chi = M rho with rho ~ exp(-rho^dag rho)
    (the heat bath's source), both solves from x0 = 0 to the workload's
    tolerance, timed with CUDA events on the current stream."""
    import math
    import torch
    from paper_2210_06874_gb300 import hmc, synth
    V, Nt = params.V, params.Nt
    rho = torch.from_numpy(synth.complex_gaussian(seed + 77, Nt, V) / math.sqrt(2.0)).to(dev)
    chi = ctx.apply_M(phi, rho, prec=hmc.PREC_FP64)
    stream = torch.cuda.current_stream()
    res = {}
    for name, prec in (("mixed", hmc.PREC_MIXED), ("fp64", hmc.PREC_FP64)):
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        x, st = ctx.cg_solve(phi, chi, tol=params.cg_tol, max_iter=params.cg_max_iter,
                             prec=prec, allow_not_converged=True)
        e.record(stream)
        e.synchronize()
        res[name] = {"ms": s.elapsed_time(e), "iterations": st.iterations,
                     "reliable_updates": st.reliable_updates,
                     "true_residual": st.true_residual, "status": st.status, "x": x}
    xm, x64 = res["mixed"].pop("x"), res["fp64"].pop("x")
    res["solution_rel_diff"] = float(torch.linalg.vector_norm(xm - x64) /
                                     torch.linalg.vector_norm(x64))
    res["chi"] = chi
    return res


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2210_06874_gb300 import build_lib, hmc, synth

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    build_lib.build()
    name = args.workload
    w, params, prec = workload_params(name, args.precision)
    if args.n_md is not None:
        params.n_md = args.n_md
    params.integrator = 1 if args.integrator == "omelyan" else 0
    if args.hb_inner > 0:
        params.hb_inner, params.hb_gamma = args.hb_inner, args.hb_gamma
    tuned = None
    if prec == "mixed" and args.operand_mode is not None:
        params.operand_mode = args.operand_mode
    if prec == "mixed" and not args.no_tune:
        from paper_2210_06874_gb300 import autotune
        if args.operand_mode is None:
            # mass preconditioning on the mixed path runs on split-K tiles
            params = autotune.tune(params, modes=(5,) if args.hb_inner > 0 else None)
        params = autotune.tune_ru(params)
        tuned = {"team_ctas": params.team_ctas, "inner_ctas": params.inner_ctas,
                 "tile_slices": params.tile_slices, "operand_mode": params.operand_mode,
                 "ru_delta": params.ru_delta}
    ctx = hmc.Context(params)
    V, Nt = params.V, params.Nt
    dev = torch.device("cuda", local_rank)
    phi = torch.from_numpy(synth.start_field(name)).to(dev)
    seed = w["seed"]
    n_therm = args.therm if args.therm is not None else THERM.get(name, 10)
    traj = 0
    for _ in range(n_therm + args.warmup):
        ctx.trajectory(phi, seed, traj, rank, allow_not_converged=True)
        traj += 1
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2
    flush_acc = torch.empty((), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    phi_start = phi.clone()   # the e2e leg replays the same trajectories from here
    traj_start = traj
    clocks.start()
    t_wall = time.perf_counter()
    total_ms, outs = 0.0, []
    for _ in range(args.steps):
        flush_l2(flush, flush_acc)          # evict L2 between timed trajectories
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        out = ctx.trajectory(phi, seed, traj, rank, allow_not_converged=True)
        e.record(stream)
        e.synchronize()
        total_ms += s.elapsed_time(e)
        outs.append(out)
        traj += 1
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    value, total_ms = aggregate_rate(total_ms, args.steps, world, dist, dev)
    if world > 1:
        dist.barrier()
    ms_per_step = total_ms / args.steps

    # end to end through the public API with host buffers: pinned phi in,
    # trajectory, phi and the trajectory record back to the host.  The chain
    # is deterministic (counter-based generator), so starting again from the
    # field at the start of the timed region with the same trajectory
    # indices repeats exactly the timed trajectories (same CG work).
    phi_host = torch.empty((Nt, V), dtype=torch.float64, pin_memory=True)
    phi_host.copy_(phi_start.cpu())
    back = torch.empty_like(phi_host)
    torch.cuda.synchronize()
    e2e_steps = args.steps
    traj = traj_start
    e2e_ms = 0.0
    for _ in range(e2e_steps):
        flush_l2(flush, flush_acc)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        phi.copy_(phi_host, non_blocking=True)
        out = ctx.trajectory(phi, seed, traj, rank, allow_not_converged=True)
        back.copy_(phi, non_blocking=True)
        stream.synchronize()
        phi_host.copy_(back)
        e.record(stream)
        e.synchronize()
        e2e_ms += s.elapsed_time(e)
        traj += 1
    e2e_ms /= e2e_steps
    h2d = Nt * V * 8
    d2h = Nt * V * 8 + 8 * 16

    # the plain FP64 GPU path on the same field and source (mixed runs only)
    n_solves = (2 * params.n_md if params.integrator == 1 else params.n_md) + 1
    cmp = None
    if prec == "mixed" and not args.no_fp64_arm:
        cmp = fp64_vs_mixed_solve(ctx, params, phi, seed, dev)
    chi_np = cmp.pop("chi").cpu().numpy() if cmp else None

    # roofline of the dominant (only) kernel: the persistent trajectory launch
    peaks, peaks_kind = load_peaks()
    mean_iters = statistics.mean(o.cg_iterations for o in outs)
    n_app = statistics.mean(applies_per_traj(o, params.n_md) for o in outs)
    flop = n_app * flops_per_apply(V, Nt)
    byts = n_app * apply_bytes(V, Nt, prec)
    achieved = flop / (ms_per_step * 1e-3) / 1e12
    hbm_peak = peaks.get("hbm_gbs", FALLBACK["hbm_gbs"])
    traffic_it, traffic_src = committed_traffic(name, "per-cg-iteration")
    traffic = traffic_it * mean_iters if traffic_it is not None else None
    hbm = {"achieved_gbs": byts / (ms_per_step * 1e-3) / 1e9, "peak_gbs": hbm_peak,
           "algorithmic_bytes": byts,
           "bytes_per_application": apply_bytes(V, Nt, prec),
           "peak_source": "%s STREAM-style copy" % peaks_kind}
    hbm["frac"] = hbm["achieved_gbs"] / hbm_peak
    if prec == "fp64":
        peak = measure_dgemm_tflops(torch)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": "measured cuBLAS DGEMM 4096^3 on this GPU (FP64 ALU peak)"}
    elif params.operand_mode == 3:
        peak, sms, mhz = fp32_fma_tflops(torch, dev)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": "FP32 FMA rate from unit counts: %d SMs (device attribute) x "
                               "128 lanes x 2 flop x %.0f MHz (the CUDA-core cluster mode runs "
                               "on one cluster)" % (sms, mhz)}
    else:
        peak = peaks.get("bf16_tflops_sustained", FALLBACK["bf16_tflops_sustained"])
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": "%s bf16 dense sustained (fp16 has the same rate)" % peaks_kind}
    roof["flop_per_application"] = flops_per_apply(V, Nt)
    roof["applications_per_launch"] = n_app
    roof["traffic_source"] = traffic_src
    roof["hbm"] = hbm
    line = {
        "metric": METRIC, "value": value, "unit": "trajectories/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": ("f64" if prec == "fp64" else
                  "f32 (f64 residuals)" if params.operand_mode == 3 else
                  "f16-split/f32 (f64 residuals)"),
        "data": "synthetic",
        "config": {"workload": name, "precision": prec, "L": w["L"], "V": V, "Nt": Nt,
                   "U": w["U"], "beta": w["beta"], "n_md": params.n_md,
                   "integrator": args.integrator,
                   "cg_tol": params.cg_tol, "thermalisation_trajectories": n_therm,
                   "l2": "flushed (256 MB write + read sweep) between timed trajectories",
                   "parallelism": "replicas (one chain per GPU)",
                   "launch_shape": tuned or "automatic"},
        "m_applications_per_s": world * n_app / (ms_per_step * 1e-3),
        "cg_iterations_per_traj": mean_iters,
        "cg_solves_per_traj": statistics.mean(o.cg_solves for o in outs),
        "cg_iterations_per_s": world * mean_iters / (ms_per_step * 1e-3),
        "acceptance": statistics.mean(o.accept for o in outs),
        "mean_abs_dH": statistics.mean(abs(o.dH) for o in outs),
        "max_true_residual": max(o.max_true_residual for o in outs),
        "e2e": {"value": world / (e2e_ms * 1e-3), "unit": "trajectories/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "how": "the timed trajectories again (same start field and indices), "
                       "phi from pinned host memory in and back every trajectory"},
        "gpu_launches": args.steps,
        "roofline": roof,
        "clocks": clk,
        "wall_s_timed_region": wall,
    }
    if args.hb_inner > 0:
        line["config"]["mass_preconditioning"] = {"hb_gamma": args.hb_gamma,
                                                  "hb_inner": args.hb_inner}
        line["cg_solves_outer_per_traj"] = statistics.mean(o.cg_solves_outer for o in outs)
        line["cg_iterations_outer_per_traj"] = statistics.mean(o.cg_iterations_outer
                                                               for o in outs)
    if cmp:
        t64 = cmp["fp64"]["ms"] * 1e-3 * n_solves
        cmp["fp64_trajectories_per_s_est"] = 1.0 / t64
        cmp["mixed_over_fp64_trajectories"] = value / world * t64
        cmp["mixed_over_fp64_solve"] = cmp["fp64"]["ms"] / cmp["mixed"]["ms"]
        cmp["how"] = ("one solve of the thermalised field's heat-bath source chi = M rho from "
                      "x0 = 0 on each path, same tolerance; the FP64 trajectory estimate is "
                      "%d such solves (the plain FP64 trajectory starts every solve from zero)"
                      % n_solves)
        line["fp64_arm"] = cmp
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        phi_np = phi.cpu().numpy()
        if V >= 288 and cmp:
            # an oracle trajectory takes minutes to hours here: time its CG
            # iterations on a bounded sample and count them by the FP64 path
            line["cpu_baseline"] = cpu_oracle_rate_by_iterations(
                name, phi_np, chi_np, args.cpu_sample_s, cmp["fp64"]["iterations"], n_solves)
            line["cpu_baseline"]["single_thread"] = cpu_oracle_rate_by_iterations(
                name, phi_np, chi_np, min(args.cpu_sample_s, 10.0), cmp["fp64"]["iterations"],
                n_solves, single_thread=True)
        else:
            hbk = (args.hb_gamma, args.hb_inner) if args.hb_inner > 0 else None
            line["cpu_baseline"] = cpu_oracle_rate(name, prec, args.cpu_sample_s,
                                                   phi_np=phi_np, integrator=args.integrator,
                                                   n_md=params.n_md, hb=hbk)
            if not hbk:
                line["cpu_baseline"]["single_thread"] = cpu_oracle_rate_single_thread(
                    name, prec, min(args.cpu_sample_s, 10.0), phi_np=phi_np,
                    integrator=args.integrator, n_md=params.n_md)
    if world == 1 and name == "l24_nt96" and prec == "mixed" and not args.no_batch_line:
        # the batched workload against the plain FP64 GPU path, in the same line
        line["batch256"] = batch_summary(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def apply_bytes(V, Nt, prec):
    """Algorithmic HBM bytes of one application: E once (FP64, or its FP16
    hi/lo split), the input and output vectors, the phase field phi and the
    phase table exp(i phi) written and read once."""
    N = V * Nt
    if prec == "fp64":
        return 8.0 * V * V + 16.0 * N * 2 + 8.0 * N + 16.0 * N * 2
    return 4.0 * V * V + 8.0 * N * 2 + 8.0 * N + 8.0 * N * 2


def run_apply(args):
    """M-applications/s of hmc_apply_M on the workload's lattice."""
    import torch
    from paper_2210_06874_gb300 import build_lib, hmc, synth

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    build_lib.build()
    name = args.workload
    w, params, prec = workload_params(name, args.precision)
    V, Nt = params.V, params.Nt
    dev = torch.device("cuda", local_rank)
    phi = torch.from_numpy(synth.gaussian_field(w["seed"], Nt, V, w["beta"] / Nt * w["U"],
                                                scale=0.5)).to(dev)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    p = hmc.PREC_FP64 if prec == "fp64" else hmc.PREC_MIXED
    psi = torch.from_numpy(synth.complex_gaussian(w["seed"] + 1, Nt, V)).to(dev).to(dt)
    out = torch.empty_like(psi)
    tried = {}
    if args.operand_mode is not None:
        params.operand_mode = args.operand_mode
    elif prec == "mixed" and not args.no_tune:
        # the standalone tile kinds (site-major 1, slice-major 4, split-K 5),
        # each timed on a few applications before the timed region
        best = None
        for mode in (1, 4, 5):
            try:
                c = hmc.Context(dataclasses.replace(params, operand_mode=mode))
            except hmc.HmcError:
                continue
            try:
                for _ in range(3):
                    c.apply_M(phi, psi, out, prec=p)
                g0 = torch.cuda.CUDAGraph()
                torch.cuda.synchronize()
                with torch.cuda.graph(g0):
                    for _ in range(10):
                        c.apply_M(phi, psi, out, prec=p)
                g0.replay()
                s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record()
                g0.replay()
                e0.record()
                e0.synchronize()
                tried[mode] = s0.elapsed_time(e0) / 10
                del g0
            except hmc.HmcError:
                continue
            finally:
                c.close()
            if best is None or tried[mode] < tried[best]:
                best = mode
        if best is not None:
            params.operand_mode = best
    ctx = hmc.Context(params)
    for _ in range(args.warmup):
        ctx.apply_M(phi, psi, out, prec=p)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    flush_acc = torch.empty((), dtype=torch.float32, device=dev)
    # the applications of a step, captured once through the C ABI into a CUDA
    # graph: its replay times the GPU work without the per-call host cost
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph):
        for _ in range(args.applies):
            ctx.apply_M(phi, psi, out, prec=p)
    graph.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    total_ms = 0.0
    for _ in range(args.steps):
        flush_l2(flush, flush_acc)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        graph.replay()
        e.record(stream)
        e.synchronize()
        total_ms += s.elapsed_time(e)
    clk = clocks.stop()
    # the same applications called one by one from Python (host-bound for
    # small lattices)
    flush_l2(flush, flush_acc)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(args.applies):
        ctx.apply_M(phi, psi, out, prec=p)
    e.record(stream)
    e.synchronize()
    eager_ms = s.elapsed_time(e) / args.applies
    e2e_ms, e2e_in, e2e_out = e2e_host_calls(
        torch, stream, psi, out, lambda: ctx.apply_M(phi, psi, out, prec=p), args.applies)
    n = args.steps * args.applies
    per_ms = total_ms / n
    flop = flops_per_apply(V, Nt)
    byts = apply_bytes(V, Nt, prec)
    peaks, kind = load_peaks()
    if prec == "fp64":
        peak = measure_dgemm_tflops(torch)
        roof = {"bound": "alu", "achieved": flop / (per_ms * 1e-3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "peak_source": "measured cuBLAS DGEMM 4096^3"}
    else:
        peak = peaks.get("bf16_tflops", FALLBACK["bf16_tflops"])
        roof = {"bound": "tensor", "achieved": flop / (per_ms * 1e-3) / 1e12, "peak": peak,
                "unit": "TFLOP/s",
                "peak_source": "%s bf16 dense burst (fp16 has the same rate)" % kind}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None
    roof["hbm"] = {"achieved_gbs": byts / (per_ms * 1e-3) / 1e9,
                   "peak_gbs": peaks.get("hbm_gbs", FALLBACK["hbm_gbs"]),
                   "algorithmic_bytes": byts}
    roof["hbm"]["frac"] = roof["hbm"]["achieved_gbs"] / roof["hbm"]["peak_gbs"]
    line = {"metric": METRIC, "value": 1e3 / per_ms, "unit": "M-applications/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else "f16-split/f32",
            "data": "synthetic",
            "config": {"workload": name, "mode": "apply", "precision": prec, "V": V, "Nt": Nt,
                       "applies_per_step": args.applies,
                       "operand_mode": params.operand_mode,
                       "operand_modes_tried_ms_per_call": {str(k): v for k, v in tried.items()}
                       or None,
                       "timing": "one CUDA-graph replay of the step's C-ABI calls",
                       "l2": "flushed (256 MB write + read sweep) between timed steps"},
            "per_call_from_python_us": eager_ms * 1e3,
            "e2e": {"value": 1e3 / e2e_ms, "unit": "M-applications/s",
                    "h2d_bytes_per_step": e2e_in, "d2h_bytes_per_step": e2e_out,
                    "how": "per call: psi from pinned host memory in, hmc_apply_M, the "
                           "result back (the field phi stays on the device)"},
            "gpu_launches": n * 2 if prec != "fp64" else n * 2,
            "roofline": roof, "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_apply_rate(name, args.cpu_sample_s)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_cg(args):
    """Microseconds per FP32 iteration of the mixed CG (two applications, two
    team sums and the vector updates) on the workload's lattice, in the
    autotuned (or --operand-mode) launch shape: the difference of two solves
    of cg_iters and cg_iters / 4 iterations (tolerance never met, reliable
    updates off), so the FP64 residual at the end of a solve cancels.
    value = M-applications/s inside the CG; the FP64 path's seconds per CG
    iteration on the same problem beside it."""
    import torch
    from paper_2210_06874_gb300 import build_lib, hmc, synth

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    build_lib.build()
    name = args.workload
    w, params, _ = workload_params(name, "mixed")
    if args.operand_mode is not None:
        params.operand_mode = args.operand_mode
    elif not args.no_tune:
        from paper_2210_06874_gb300 import autotune
        params = autotune.tune(params)
    params.ru_delta = 1e-30
    params.ru_every = 1 << 30
    ctx = hmc.Context(params)
    V, Nt = params.V, params.Nt
    dev = torch.device("cuda", local_rank)
    phi = torch.from_numpy(synth.gaussian_field(w["seed"], Nt, V, w["beta"] / Nt * w["U"],
                                                scale=0.3)).to(dev)
    chi = torch.from_numpy(synth.complex_gaussian(w["seed"] + 1, Nt, V)).to(dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    flush_acc = torch.empty((), dtype=torch.float32, device=dev)
    n_long, n_short = args.cg_iters, max(1, args.cg_iters // 4)

    def solve_ms(prec, iters):
        flush_l2(flush, flush_acc)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        _, st = ctx.cg_solve(phi, chi, tol=1e-300, max_iter=iters, prec=prec,
                             allow_not_converged=True)
        e.record(stream)
        e.synchronize()
        assert st.iterations == iters, (st.iterations, iters)
        return s.elapsed_time(e)

    for _ in range(max(1, args.warmup)):
        solve_ms(hmc.PREC_MIXED, n_short)
    clocks = ClockSampler(local_rank)
    clocks.start()
    per_it = []
    for _ in range(args.steps):
        per_it.append((solve_ms(hmc.PREC_MIXED, n_long) - solve_ms(hmc.PREC_MIXED, n_short)) /
                      (n_long - n_short))
    clk = clocks.stop()
    ms_it = statistics.median(per_it)
    n64 = max(8, n_long // 20)
    # end to end: chi from pinned host memory in, the long solve, x back
    xbuf = torch.empty_like(chi)

    def long_solve():
        ctx.cg_solve(phi, chi, tol=1e-300, max_iter=n_long, prec=hmc.PREC_MIXED, x=xbuf,
                     allow_not_converged=True)
    e2e_ms, e2e_in, e2e_out = e2e_host_calls(torch, stream, chi, xbuf, long_solve, 1)
    ms64 = (solve_ms(hmc.PREC_FP64, 2 * n64) - solve_ms(hmc.PREC_FP64, n64)) / n64
    peaks, kind = load_peaks()
    flop = 2 * flops_per_apply(V, Nt)
    byts = 2 * apply_bytes(V, Nt, "mixed")
    peak = peaks.get("bf16_tflops", FALLBACK["bf16_tflops"])
    hbm_peak = peaks.get("hbm_gbs", FALLBACK["hbm_gbs"])
    achieved = flop / (ms_it * 1e-3) / 1e12
    traffic_it, traffic_src = committed_traffic(name, "per-cg-iteration")
    line = {"metric": METRIC, "value": 2e3 / ms_it, "unit": "M-applications/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(per_it) * (n_long - n_short),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f16-split/f32", "data": "synthetic",
            "config": {"workload": name, "mode": "cg", "V": V, "Nt": Nt,
                       "iterations": [n_short, n_long],
                       "launch_shape": {"team_ctas": params.team_ctas,
                                        "inner_ctas": params.inner_ctas,
                                        "tile_slices": params.tile_slices,
                                        "operand_mode": params.operand_mode},
                       "field": "phi ~ 0.3 N(0, delta U), chi complex Gaussian",
                       "l2": "flushed (256 MB write + read sweep) before every solve"},
            "us_per_cg_iteration": 1e3 * ms_it,
            "fp64_us_per_cg_iteration": 1e3 * ms64,
            "e2e": {"value": 2e3 * n_long / e2e_ms, "unit": "M-applications/s",
                    "h2d_bytes_per_step": e2e_in, "d2h_bytes_per_step": e2e_out,
                    "how": "one solve of the longer length with chi in from pinned host "
                           "memory and x back (its FP64 set-up and final residual "
                           "included, unlike the value)"},
            "gpu_launches": 2 * args.steps,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": (traffic_it * 1.0) if traffic_it is not None else None,
                         "traffic_source": traffic_src,
                         "flop_per_iteration": flop,
                         "peak_source": "%s bf16 dense burst (fp16 has the same rate)" % kind,
                         "hbm": {"achieved_gbs": byts / (ms_it * 1e-3) / 1e9,
                                 "peak_gbs": hbm_peak, "algorithmic_bytes": byts,
                                 "frac": byts / (ms_it * 1e-3) / 1e9 / hbm_peak}},
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_batch(args, emit=True):
    """Batched workload: many chains of uneven size, one persistent launch per
    trajectory of every chain (hmc_batch_trajectory); value = aggregate
    trajectories/s.  Also times the same chains as a loop of single-chain
    hmc_trajectory launches (each using the whole GPU)."""
    import torch
    from paper_2210_06874_gb300 import build_lib, hmc, synth

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    build_lib.build()
    n = args.chains
    specs = synth.batch256(n_chains=n)
    plist = [hmc.Params(L=c["L"], Nt=c["Nt"], kappa=c["kappa"], U=c["U"], beta=c["beta"],
                        n_md=c["n_md"], traj_length=c["traj_length"], cg_tol=c["cg_tol"],
                        cg_max_iter=200000, precision=hmc.PREC_MIXED) for c in specs]
    shapes = {}
    if not args.no_tune:
        from paper_2210_06874_gb300 import autotune
        # one-CTA shapes, and cluster teams for the chains that would
        # otherwise finish last
        tuned = autotune.batch_shapes(plist, csize=args.batch_team)
        for p in tuned:
            # per class: the shape of its one-CTA chains (or, if all of them
            # are teams, the team shape) and how many of its chains are teams
            key = "L%d_Nt%d" % (p.L, p.Nt)
            ent = shapes.setdefault(key, {"chains": 0, "team_chains": 0})
            ent["chains"] += 1
            if p.team_ctas > 1:
                ent["team_chains"] += 1
                ent.setdefault("team", {"team_ctas": p.team_ctas,
                                        "tile_slices": p.tile_slices,
                                        "operand_mode": p.operand_mode,
                                        "ru_delta": p.ru_delta})
            else:
                ent.setdefault("one_cta", {"tile_slices": p.tile_slices,
                                           "operand_mode": p.operand_mode,
                                           "ru_delta": p.ru_delta})
        loop_params = [autotune.tune_ru(autotune.tune(p)) for p in plist[:args.loop_chains]]
        plist = tuned
    else:
        loop_params = plist[:args.loop_chains]
    b = hmc.Batch(plist)
    dev = torch.device("cuda", local_rank)
    phi = torch.zeros(b.total, dtype=torch.float64, device=dev)   # cold start
    seed = synth.BASE_SEED + 3 + 1000 * rank
    traj = 0
    n_therm = args.therm if args.therm is not None else 2
    for _ in range(n_therm + args.warmup):
        b.trajectory(phi, seed, traj, allow_failure=True)
        traj += 1
    clocks = ClockSampler(local_rank)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    phi_start, traj_start = phi.clone(), traj   # the e2e leg replays the timed steps
    clocks.start()
    total_ms, outs = 0.0, []
    for _ in range(args.steps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        o = b.trajectory(phi, seed, traj, allow_failure=True)
        e.record(stream)
        e.synchronize()
        total_ms += s.elapsed_time(e)
        outs.extend(o)
        traj += 1
    clk = clocks.stop()
    value = world * n * args.steps / (total_ms * 1e-3)
    # end to end through the public API with host buffers: every chain's
    # field in from pinned host memory, one batched trajectory, the fields
    # back (the per-chain records come back inside the call)
    # (the same steps again from the same fields and trajectory indices: the
    # chains are deterministic, so the work is the timed work)
    phi_end = phi.clone()
    phi_host = torch.empty(b.total, dtype=torch.float64, pin_memory=True)
    phi_host.copy_(phi_start.cpu())
    back = torch.empty_like(phi_host)
    torch.cuda.synchronize()
    e2e_steps = args.steps
    t_e2e = traj_start
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(e2e_steps):
        phi.copy_(phi_host, non_blocking=True)
        b.trajectory(phi, seed, t_e2e, allow_failure=True)
        back.copy_(phi, non_blocking=True)
        stream.synchronize()
        phi_host.copy_(back)
        t_e2e += 1
    e.record(stream)
    e.synchronize()
    e2e_value = world * n / (s.elapsed_time(e) / e2e_steps * 1e-3)
    phi.copy_(phi_end)
    e2e_bytes = b.total * 8
    # loop of single-chain launches over the same chains (first K_loop chains)
    n_loop = min(n, args.loop_chains)
    loop_ms = 0.0
    if n_loop > 0:
        ctxs = [hmc.Context(p) for p in loop_params[:n_loop]]
        fields = [b.view(phi, i).clone() for i in range(n_loop)]
        for i, c in enumerate(ctxs):
            c.trajectory(fields[i], seed, traj, chain=i, allow_not_converged=True)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        for i, c in enumerate(ctxs):
            c.trajectory(fields[i], seed, traj + 1, chain=i, allow_not_converged=True)
        e.record(stream)
        e.synchronize()
        loop_ms = s.elapsed_time(e)
    # the plain FP64 GPU path on the first chains, one launch per chain, same
    # tolerance and fields
    n64 = min(n, args.loop_chains_fp64)
    loop64_ms = 0.0
    if n64 > 0:
        p64 = [hmc.Params(**{**plist[i].__dict__, "precision": hmc.PREC_FP64,
                             "team_ctas": 0, "inner_ctas": 0, "tile_slices": 0,
                             "operand_mode": 0}) for i in range(n64)]
        ctxs64 = [hmc.Context(p) for p in p64]
        fields64 = [b.view(phi, i).clone() for i in range(n64)]
        for i, c in enumerate(ctxs64):
            c.trajectory(fields64[i], seed, traj, chain=i, allow_not_converged=True)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        for i, c in enumerate(ctxs64):
            c.trajectory(fields64[i], seed, traj + 1, chain=i, allow_not_converged=True)
        e.record(stream)
        e.synchronize()
        loop64_ms = s.elapsed_time(e)
    # the plain FP64 GPU path over the whole workload, estimated per class:
    # one FP64 trajectory of the first chain of every (L, Nt) class from its
    # current field (same cg_tol), weighted by the class's chain count
    classes = {}
    for i, p in enumerate(plist):
        classes.setdefault((p.L, p.Nt), []).append(i)
    per_class = []
    est64_ms = 0.0
    if not args.no_fp64_arm:
        for (L_, Nt_), idx in sorted(classes.items()):
            i = idx[0]
            pc = hmc.Params(**{**plist[i].__dict__, "precision": hmc.PREC_FP64,
                               "team_ctas": 0, "inner_ctas": 0, "tile_slices": 0,
                               "operand_mode": 0})
            c64 = hmc.Context(pc)
            f = b.view(phi, i).clone()
            torch.cuda.synchronize()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            o64 = c64.trajectory(f, seed, traj + 3, chain=i, allow_not_converged=True)
            e.record(stream)
            e.synchronize()
            ms = s.elapsed_time(e)
            est64_ms += ms * len(idx)
            per_class.append({"L": L_, "Nt": Nt_, "chains": len(idx), "sampled_chain": i,
                              "fp64_ms": ms, "cg_iterations": o64.cg_iterations})
            del c64
    # the mixed loop over exactly those chains
    loop_mixed_same_ms = 0.0
    if n64 > 0 and n_loop >= n64:
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        for i, c in enumerate(ctxs[:n64]):
            c.trajectory(fields[i], seed, traj + 2, chain=i, allow_not_converged=True)
        e.record(stream)
        e.synchronize()
        loop_mixed_same_ms = s.elapsed_time(e)
    sizes = [(p.L, p.Nt) for p in plist]
    flop = sum((applies_per_traj(o, plist[i % n].n_md)) * flops_per_apply(plist[i % n].V,
                                                                         plist[i % n].Nt)
               for i, o in enumerate(outs)) / args.steps
    peaks, kind = load_peaks()
    peak = peaks.get("bf16_tflops_sustained", FALLBACK["bf16_tflops_sustained"])
    achieved = flop / (total_ms / args.steps * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "trajectories/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f16-split/f32 (f64 residuals)", "data": "synthetic",
        "config": {"workload": "batch%d" % n, "precision": "mixed", "chains": n,
                   "L_set": sorted(set(p.L for p in plist)),
                   "Nt_set": sorted(set(p.Nt for p in plist)),
                   "thermalisation_trajectories": n_therm,
                   "step": "one trajectory of every chain in one persistent launch (CUDA graph)",
                   "shape_by_autotuner": shapes or "automatic",
                   "l2": "inputs (all chains' fields and workspaces) exceed one trajectory's "
                         "reuse window; no flush"},
        "loop_of_single_chain_launches": {
            "chains": n_loop, "ms": loop_ms,
            "trajectories_per_s": n_loop / (loop_ms * 1e-3) if loop_ms else None},
        "fp64_whole_workload_est": {
            "trajectories_per_s": n / (est64_ms * 1e-3) if est64_ms else None,
            "mixed_batched_over_fp64": value / (n / (est64_ms * 1e-3)) if est64_ms else None,
            "how": "plain FP64 GPU path (hmc_trajectory, precision FP64, one chain per "
                   "launch, same cg_tol 1e-10 FP64 true residual): one trajectory of one "
                   "chain per (L, Nt) class from its field after the timed steps, "
                   "times the class's chain count, summed",
            "classes": per_class} if est64_ms else None,
        "loop_of_single_chain_launches_fp64": {
            "chains": n64, "ms": loop64_ms,
            "trajectories_per_s": n64 / (loop64_ms * 1e-3) if loop64_ms else None,
            "path": "plain FP64 GPU path (hmc_trajectory, precision FP64), same cg_tol",
            "mixed_same_chains_ms": loop_mixed_same_ms or None},
        "acceptance": statistics.mean(o.accept for o in outs),
        "cg_iterations_per_traj": statistics.mean(o.cg_iterations for o in outs),
        "max_true_residual": max(o.max_true_residual for o in outs),
        "statuses": sorted(set(o.status for o in outs)),
        "e2e": {"value": e2e_value, "unit": "trajectories/s",
                "h2d_bytes_per_step": e2e_bytes,
                "d2h_bytes_per_step": e2e_bytes + n * 16 * 8},   # + 16 doubles per chain record
        "gpu_launches": args.steps,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_source": "%s bf16 dense sustained (fp16 has the same rate)" % kind},
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        flds = {pc["sampled_chain"]: b.view(phi, pc["sampled_chain"]).cpu().numpy()
                for pc in per_class}
        line["cpu_baseline"] = cpu_oracle_batch_rate(args.chains, args.cpu_sample_s,
                                                     per_class or None, flds)
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    return line


def batch_summary(args):
    """The batched workload's comparison, run after the default single-chain
    line on one GPU: the batched mixed form against the plain FP64 GPU path
    over the same 256 chains (a few steps; failures are reported, not
    raised)."""
    import copy
    b_args = copy.copy(args)
    # the standalone batched line's schedule (2 thermalisation trajectories
    # and the bench's warm-up ones from a cold start, then 3 timed): the
    # chains grow more expensive as they thermalise, so both report the same
    b_args.steps, b_args.therm = 3, None
    b_args.cpu_sample_s = min(args.cpu_sample_s, 10.0)
    try:
        d = run_batch(b_args, emit=False)
    except Exception as e:   # an extra of the default line: never fail the bench on it
        return {"workload": "batch%d" % args.chains, "unavailable": str(e)[:300]}
    f = d.get("fp64_whole_workload_est") or {}
    out = {"workload": d["config"]["workload"], "metric": "aggregate trajectories/s",
           "value": d["value"], "unit": d["unit"], "steps": d["steps"],
           "ms_per_step": d["ms_per_step"], "e2e": d["e2e"],
           "fp64_whole_workload_trajectories_per_s": f.get("trajectories_per_s"),
           "mixed_batched_over_fp64": f.get("mixed_batched_over_fp64"),
           "fp64_how": f.get("how"), "statuses": d["statuses"],
           "cg_iterations_per_traj": d["cg_iterations_per_traj"],
           "roofline": d["roofline"], "clocks": d["clocks"],
           "loop_of_single_chain_launches": d["loop_of_single_chain_launches"]}
    if "cpu_baseline" in d:
        out["cpu_baseline"] = {k: d["cpu_baseline"][k] for k in ("value", "unit", "cores", "kind")
                               if k in d["cpu_baseline"]}
    return out


def run_brs(args):
    """Eq. (2.2) operator (mixed differencing, sparse stencil) on the paper's
    largest lattice, L = 102 (20,808 sites): M-applications/s against the HBM
    roofline.  Algorithmic bytes per site-slice: input vector, phase table and
    output once each (FP32: 24 B, FP64: 48 B)."""
    import torch
    from paper_2210_06874_gb300 import build_lib, hmc, synth

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    build_lib.build()
    L, Nt, beta, kappa = args.brs_L, args.brs_Nt, 0.125 * args.brs_Nt, 1.0
    V = 2 * L * L
    N = V * Nt
    dev = torch.device("cuda", local_rank)
    prec = args.precision or "mixed"
    phi = torch.from_numpy(synth.gaussian_field(7, Nt, V, 0.125 * 4.0, scale=0.5)).to(dev)
    c64, c32 = hmc.brs_phases(L, Nt, phi)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    cis = c64 if prec == "fp64" else c32
    psi = torch.from_numpy(synth.complex_gaussian(8, Nt, V)).to(dev).to(dt)
    out = torch.empty_like(psi)
    for _ in range(args.warmup):
        hmc.apply_brs(L, Nt, beta / Nt * kappa, cis, psi, out)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    flush_acc = torch.empty((), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local_rank)
    torch.cuda.synchronize()
    clocks.start()
    times = []
    for _ in range(args.steps):
        for _ in range(args.applies):
            flush_l2(flush, flush_acc)     # every application starts with a cold L2
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            hmc.apply_brs(L, Nt, beta / Nt * kappa, cis, psi, out)
            e.record(stream)
            e.synchronize()
            times.append(s.elapsed_time(e))
    clk = clocks.stop()
    per_ms = statistics.median(times)
    e2e_ms, e2e_in, e2e_out = e2e_host_calls(
        torch, stream, psi, out, lambda: hmc.apply_brs(L, Nt, beta / Nt * kappa, cis, psi, out),
        args.applies)
    bpe = 48.0 if prec == "fp64" else 24.0
    byts = bpe * N
    peaks, kind = load_peaks()
    hbm = peaks.get("hbm_gbs", FALLBACK["hbm_gbs"])
    achieved = byts / (per_ms * 1e-3) / 1e9
    line = {"metric": METRIC, "value": 1e3 / per_ms, "unit": "M-applications/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": "brs_l%d_nt%d" % (L, Nt), "operator": "Eq. (2.2) stencil",
                       "V": V, "Nt": Nt, "applies_per_step": args.applies,
                       "l2": "flushed (256 MB write + read sweep) before every application; median"},
            "gpu_launches": args.steps * args.applies,
            "e2e": {"value": 1e3 / e2e_ms, "unit": "M-applications/s",
                    "h2d_bytes_per_step": e2e_in, "d2h_bytes_per_step": e2e_out,
                    "how": "per call: psi from pinned host memory in, hmc_apply_brs, the "
                           "result back (the phase table stays on the device)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": None,
                         "algorithmic_bytes_per_apply": byts,
                         "peak_source": "%s STREAM-style copy" % kind},
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.mode == "brs" and args.impl == "ours":
        run_brs(args)
        return
    if args.workload.startswith("batch") and args.impl == "ours":
        run_batch(args)
        return
    if args.mode == "apply" and args.impl == "ours":
        run_apply(args)
        return
    if args.mode == "cg" and args.impl == "ours":
        run_cg(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
