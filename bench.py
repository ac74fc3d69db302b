#!/usr/bin/env python
"""Benchmark of the sparse-SYK OTOC hot path: H psi at N = 64.

Workload (the N = 64 configuration the headline metric is quoted on): one
sparse-SYK realisation with N = 64 Majoranas, k = 4 (Bernoulli mask, ~256
terms), Jordan-Wigner representation, one parity block of D = 2^31
amplitudes (complex64: 16 GiB per vector).  A step is one H_UU psi through
syk_apply_H with psi and Phi resident in HBM (both far larger than the
126 MB L2, so no L2 flush is needed between steps).  The float64 variant
(complex128, 32 GiB per vector) is reported alongside.

Multi-GPU: replicas only (each rank its own realisation, no collective on the
data path); value = all ranks' term*amplitude updates / max time over ranks.

`--impl reference` times the oracle's C++/OpenMP CPU baseline (a bounded
sample of output rows of the same H psi, FP64, all host cores) instead.
"""
from __future__ import annotations

import argparse
import importlib.util
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H·ψ Gterm·amp/s at N=64 (fp32 vs fp64); OTOC realizations/s; p50/p99 latency"
UNIT = "Gterm·amp/s"
ISSUE_SLOTS_PER_TERM_AMP = 3  # 2 FP32 FMA + 1 load per term x amplitude


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="all",
                    choices=["all", "otoc-batch", "otoc-serve", "n64-otoc", "spin", "nonherm", "paper-rows", "config2"],
                    help="all: the benchmark line; otoc-batch / otoc-serve / n64-otoc / spin / nonherm: only that "
                         "leg, as its own JSON line (spin: random-field Heisenberg chain, H psi and OTOC curves; "
                         "nonherm: non-Hermitian SYK, H psi and Arnoldi OTOC curves; paper-rows: time per OTOC "
                         "curve of the paper's benchmark rows; config2: the N=32 mixed-precision error statement)")
    ap.add_argument("--rows-N", default="30,38,46", help="paper-rows: the N values (k=3, beta=0.05)")
    ap.add_argument("--rows-dense-N", default="30", help="paper-rows: N values of dense SYK rows ('' for none)")
    ap.add_argument("--N", type=int, default=64)
    ap.add_argument("--dense", action="store_true", help="H psi step on dense SYK (every quadruple) at --N")
    ap.add_argument("--k", type=float, default=4.0)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-relabel", action="store_true",
                    help="use the identity Jordan-Wigner order instead of the locality-ordered labels")
    ap.add_argument("--no-identity", action="store_true",
                    help="skip the comparison timing of the identity Jordan-Wigner order")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-l2", action="store_true")
    ap.add_argument("--no-otoc", action="store_true", help="skip the batched / served OTOC legs")
    ap.add_argument("--no-outlook", action="store_true",
                    help="skip the spin-chain and non-Hermitian H psi keys of the benchmark line")
    ap.add_argument("--n64-m", type=int, default=10, help="Krylov dimension of the N=64 end-to-end OTOC")
    ap.add_argument("--n64-two-pass", action="store_true",
                    help="N=64 OTOC: regenerate the Krylov basis in a second pass (3 vectors) instead of storing "
                         "m+1 vectors (m=10 stored: 64 s/point; m=20 two-pass: 80 s/point; m=8 stored: 100 s/point)")
    ap.add_argument("--batch-realizations", type=int, default=32)
    ap.add_argument("--batch-states", type=int, default=4)
    ap.add_argument("--batch-slots", type=int, default=4096,
                    help="batch slots (jobs live at once; the rest wait for admission)")
    ap.add_argument("--batch-N", type=int, default=0, help="batched leg: fixed N for every realisation (0: 24..36)")
    ap.add_argument("--batch-k", type=float, default=3.0, help="batched leg: k with --batch-N")
    ap.add_argument("--batch-no-plain", action="store_true",
                    help="batched leg: skip the plain FP64 single-realisation comparison")
    ap.add_argument("--no-batch-autotune", action="store_true",
                    help="batched leg: library default Krylov dimension and sync period, no autotuner")
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-tmax", type=float, default=20.0)
    ap.add_argument("--serve-dt", type=float, default=1.0)
    ap.add_argument("--spin-L", type=int, default=31, help="spin leg: qubits of the H psi chain (D = 2^L)")
    ap.add_argument("--spin-otoc-L", type=int, default=20, help="spin leg: qubits of the OTOC-curve chain")
    ap.add_argument("--spin-beta", type=float, default=0.0,
                    help="spin leg: inverse temperature of the OTOC curves (0: infinite temperature)")
    ap.add_argument("--serve-hbm-gb", type=float, default=150.0, help="served leg: device arena for live jobs")
    ap.add_argument("--serve-capacity-requests", type=int, default=0,
                    help="served leg: requests of the closed-loop capacity run (0: all of --serve-requests)")
    ap.add_argument("--serve-slots", type=int, default=256, help="served leg: jobs live at once")
    ap.add_argument("--serve-policy", default="fifo", choices=["fifo", "sjf"],
                    help="served leg: admission order (fifo, or shortest estimated work first)")
    ap.add_argument("--serve-load", type=float, default=0.75,
                    help="Poisson arrival rate as a fraction of the closed-loop capacity (all requests at t=0)")
    return ap.parse_args()


def workload_config(args, T):
    rep = ("jw, Majoranas relabelled for locality (syk_relabel_majoranas)" if not getattr(args, "no_relabel", False)
           else "jw")
    D = 1 << (args.N // 2 - 1)
    kind = f"dense SYK H·psi, N={args.N}" if getattr(args, "dense", False) else f"sparse SYK H·psi, N={args.N}, k={args.k:g}"
    return {"workload": f"{kind}, one parity block",
            "N": args.N, "k": "dense" if getattr(args, "dense", False) else args.k, "terms": T, "D": D, "rep": rep,
            "states": 1, "l2": ("inputs larger than L2 (16 GiB per vector), no flush" if D * 8 > (128 << 20)
                               else "inputs L2-resident (smaller than the 126 MB L2)")}


# The relabelling search of the benchmark Hamiltonian: 3 restarts of 3 000 000
# annealing moves (about 7 s on the host, before any timed region), the labels
# with the cheapest default plan kept (relabel_for_locality).
RELABEL = {"iterations": 3_000_000, "restarts": 3}


_relabel_cache = {}


def _relabel(syk, N, q, J, M=None):
    """relabel_for_locality with the benchmark's search, once per term list."""
    import numpy as np

    key = (N, np.asarray(q, np.int32).tobytes(), np.asarray(J, np.float64).tobytes(),
           None if M is None else np.asarray(M, np.float64).tobytes())
    if key not in _relabel_cache:
        _relabel_cache[key] = syk.relabel_for_locality(N, q, J, M=M, **RELABEL)
    return _relabel_cache[key]


def locality_terms(syk, N, q, J, args):
    """The benchmark Hamiltonian in the library's locality-ordered
    Jordan-Wigner labels (the same operator up to a unitary change of basis;
    fewer staged input tiles per output tile), unless --no-relabel."""
    if getattr(args, "no_relabel", False):
        return q, J, None
    r = _relabel(syk, N, q, J)
    return r["quads"], r["J"], {"patterns_before": r["patterns_before"], "patterns_after": r["patterns_after"],
                                "search": dict(RELABEL, seed=r["seed"], plan_costs=r["plan_costs"])}


def locality_terms_complex(syk, N, q, J, M, args):
    """The same relabelling for couplings J + iM (the library flips M with J)."""
    if getattr(args, "no_relabel", False):
        return q, J, M, None
    r = _relabel(syk, N, q, J, M)
    return r["quads"], r["J"], r["M"], {"patterns_after": r["patterns_after"], "seed": r["seed"]}


# ------------------------------------------------------------------ clocks --
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- the oracle --
def oracle_rows_rate(N, k, seconds=12.0, seed=77):
    """CPU oracle: sampled rows of H_UU psi from the definition (basis-state
    maps, numpy).  Returns (Gterm*amp/s, rows, T, threads)."""
    import numpy as np

    import syk_inputs as si
    from oracle import hamiltonian as ham

    q, J, _ = si.sample_sparse_syk(N, k, r=0)
    T = len(J)
    D = 1 << (N // 2 - 1)
    rng = np.random.default_rng(seed)

    def run(nrows):
        rows = rng.integers(0, D, nrows).astype(np.uint64)
        needed = []
        ham.rows_of_Hpsi(N, q, J, "jw", 0, rows, lambda b, m: needed.append(m.copy()) or np.zeros(len(m)))
        idx = np.unique(np.concatenate(needed))
        vals = si.philox_state(N, seed, 0, idx)  # inputs, generated outside the timed region
        lookup = lambda b, m: vals[np.searchsorted(idx, m)]
        t0 = time.perf_counter()
        ham.rows_of_Hpsi(N, q, J, "jw", 0, rows, lookup)
        return time.perf_counter() - t0

    dt = run(256)
    nrows = int(min(1 << 20, max(256, 256 * seconds / max(dt, 1e-3))))
    dt = run(nrows)
    return T * nrows / dt / 1e9, nrows, T, 1


def host_info():
    """CPU model and logical core count of this host."""
    model = "unknown"
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"cpu_model": model, "nproc": os.cpu_count()}


def cpp_rows_rate(N, k, seconds=10.0, log2R=18, seed=77):
    """C++/OpenMP CPU baseline (oracle/cpu_baseline.cpp, all host cores, FP64):
    the output rows [0, 2^log2R) of H_UU psi for the N-Majorana workload, a
    bounded sample of the full product.  Each term reads one aligned range of
    2^log2R input amplitudes, filled with seeded Gaussian values outside the
    timed region.  Returns (Gterm*amp/s, rows, T, threads, calls)."""
    import numpy as np

    import syk_inputs as si
    from oracle import cpu_baseline as cb

    q, J, _ = si.sample_sparse_syk(N, k, r=0)
    T = len(J)
    log2R = min(log2R, N // 2 - 1)
    starts = cb.row_sample_starts(N, q, J, 0, 0, log2R)
    data = {}
    for s0 in sorted(set(int(v) for v in starts)):
        rng = np.random.default_rng(seed + s0)
        data[s0] = rng.normal(size=1 << log2R) + 1j * rng.normal(size=1 << log2R)
    blocks = [data[int(v)] for v in starts]
    cb.hpsi_rows(N, q, J, 0, 0, log2R, blocks)  # warm-up
    calls, t0 = 0, time.perf_counter()
    while True:
        cb.hpsi_rows(N, q, J, 0, 0, log2R, blocks)
        calls += 1
        dt = time.perf_counter() - t0
        if dt >= seconds or calls >= 10000:
            break
    return T * (1 << log2R) * calls / dt / 1e9, 1 << log2R, T, cb.threads(), calls


def cpp_full_rates(k, Ns=(32, 40, 48), seconds=3.0):
    """Full-block H_UU psi with the C++/OpenMP baseline at each N (complex128
    vectors in host memory), a Lanczos evolve e^{-iH}psi at N=32 (m=30,
    tol 1e-12), and dense exact diagonalisation (numpy eigh of the full
    256 x 256 H) at N = 16."""
    import numpy as np

    import syk_inputs as si
    from oracle import cpu_baseline as cb
    from oracle import dynamics as dyn
    from oracle import hamiltonian as ham

    out = {}
    for N in Ns:
        q, J, _ = si.sample_sparse_syk(N, k, r=0)
        D = 1 << (N // 2 - 1)
        psi = np.random.default_rng(N).normal(size=D) + 0j
        cb.hpsi(N, q, J, 0, psi)
        calls, t0 = 0, time.perf_counter()
        while True:
            cb.hpsi(N, q, J, 0, psi)
            calls += 1
            dt = time.perf_counter() - t0
            if dt >= seconds:
                break
        out[f"N{N}"] = {"Gtermamp_s": len(J) * D * calls / dt / 1e9, "ms_per_Hpsi": dt * 1e3 / calls,
                        "terms": len(J), "D": D}
    q, J, _ = si.sample_sparse_syk(32, k, r=0)
    x = np.random.default_rng(5).normal(size=1 << 15) + 0j
    x /= np.linalg.norm(x)
    t0 = time.perf_counter()
    _, mv = cb.krylov_evolve(32, q, J, 0, 1j, x, m=30, tol=1e-12)
    out["krylov_N32"] = {"s": time.perf_counter() - t0, "matvecs": mv, "z": "i (t = 1)", "m": 30, "tol": 1e-12}
    q, J, _ = si.sample_sparse_syk(16, k, r=0)
    H = ham.dense_H(16, q, J, "jw")
    t0 = time.perf_counter()
    dyn.eig(H)
    out["ed_N16_s"] = time.perf_counter() - t0
    return out


def reference_arm(args):
    """The reference arm for this build is the oracle: its C++/OpenMP CPU
    baseline timed on all host cores, each step a bounded sample (2^18 output
    rows) of the same N = 64 H psi workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    t0 = time.perf_counter()
    vals = []
    for _ in range(max(1, args.warmup)):
        cpp_rows_rate(args.N, args.k, seconds=1.0)
    for _ in range(max(1, args.steps)):
        v, nrows, T, cores, _ = cpp_rows_rate(args.N, args.k, seconds=3.0)
        vals.append(v)
    value = statistics.median(vals)
    sample = (f"output rows [0, {nrows}) of H_UU psi (of D=2^{args.N // 2 - 1}), T={T} terms, C++/OpenMP FP64, "
              f"{cores} threads, about 3 s per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": (time.perf_counter() - t0) * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, T),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             **host_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# sources whose change invalidates the committed DRAM-traffic capture: the
# kernel, its shared helpers, the pass planner and the record layout
KERNEL_SOURCES = ("apply.cu", "tma_common.cuh", "device_common.cuh", "plan.cpp", "records.cpp", "capi.cu", "internal.h")


def plan_dram_model(syk, N, q, J):
    """DRAM bytes per H psi predicted from the pass plan: every pass reads its
    input once (its super-tiles stay in L2 for the pass's terms) and writes the
    output once, passes after the first also read the partial sum, and each
    straggler term reads its input tiles from DRAM."""
    pl = syk.plan_host(N, q, J, dtype="c64")
    D = 1 << (N // 2 - 1)
    read = write = 0
    for i, p in enumerate(pl["passes"]):
        strag = int(pl["straggler"][p["t0"]:p["t1"]].sum())
        read += 8 * D * (1 + (1 if i > 0 else 0) + strag)
        write += 8 * D
    return read, write


def measured_traffic(syk, N, q, J):
    """DRAM bytes per H psi: the plan model for this Hamiltonian times the
    ratio measured / modelled of the committed small-case ncu capture (N=56,
    1 GiB vectors), if that capture was taken on the current kernel, planner
    and record sources (else None)."""
    import hashlib

    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "matvec_c64_traffic.json")))
        h = hashlib.sha256()
        for f in KERNEL_SOURCES:
            h.update(open(os.path.join(ROOT, "paper_2311_00639_b300", "csrc", f), "rb").read())
        if rec.get("kernel_sources_sha256") != h.hexdigest():
            return None
        r, w = plan_dram_model(syk, N, q, J)
        return (r + w) * rec["measured_over_model"]
    except Exception:
        return None


# ------------------------------------------------------------- OTOC legs ----
def otoc_batched(args, syk, si, torch, rank=0):
    """Batched OTOC (bounded form of the 4096-realisation configuration):
    R realisations, N uniform in {24,...,36}, k uniform in {1,2,4,8}, beta=10,
    S typical states each, t = 0..10 in 10 segments, complex64 states with
    FP64 Lanczos scalars.  Also times the plain FP64 single-realisation path
    (syk_otoc, complex128) on the same first realisations and reports the
    complex64-vs-complex128 OTOC difference."""
    import numpy as np

    rng = np.random.default_rng(4242 + rank)
    R, S = args.batch_realizations, args.batch_states
    grid = np.linspace(0.0, 10.0, 11)
    beta = 10.0
    reals = []
    for r in range(R):
        N = int(rng.choice(np.arange(24, 37, 2)))
        k = float(rng.choice([1.0, 2.0, 4.0, 8.0]))
        if args.batch_N:  # one size for every realisation (e.g. a paper row through the batched engine)
            N, k = args.batch_N, args.batch_k
        q, J, _ = si.sample_sparse_syk(N, k, seed=700_000 + 1000 * rank + r)
        reals.append((N, q, J, syk.Terms(N, q, J, dtype="c64")))
    jobs = [(r, s) for r in range(R) for s in range(S)]
    # Krylov dimension and host sync period: picked by the library's batch
    # autotuner on a random sample of these jobs (untimed, like plan building)
    tune = None
    m, tps = 0, 16
    if not args.no_batch_autotune:
        pick = rng.choice(len(jobs), size=min(len(jobs), 64), replace=False)
        sample = [(reals[jobs[i][0]][3], reals[jobs[i][0]][0] - 1, reals[jobs[i][0]][0] - 2, beta, grid,
                   1234 + jobs[i][0], jobs[i][1]) for i in pick]
        t0 = time.perf_counter()
        tune = syk.autotune_batch(sample, dtype="c64", max_bytes=8 << 30)
        tune["tuning_s"] = time.perf_counter() - t0
        tune["sample_jobs"] = len(sample)
        m, tps = tune["m"], tune["ticks_per_sync"]
    b = syk.Batch(dtype="c64", max_slots=min(len(jobs), args.batch_slots), max_bytes=40 << 30, m=m)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    results = {}
    queue = list(enumerate(jobs))
    while queue or b.pending:
        while queue:
            tag, (r, s) = queue[0]
            N, _, _, h = reals[r]
            if not b.submit(h, N - 1, N - 2, beta, grid, 1234 + r, s, tag):
                break
            queue.pop(0)
        for res in b.run(ticks_per_sync=tps):
            results[res["tag"]] = res
    wall = time.perf_counter() - t0
    termamps = sum(results[t]["matvecs"] * reals[jobs[t][0]][3].n_terms * reals[jobs[t][0]][3].D for t in results)
    b.close()
    sizes = f"N={args.batch_N}, k={args.batch_k:g}" if args.batch_N else "N in 24..36, k in 1,2,4,8"
    out = {"workload": f"{R} realisations x {S} states, {sizes}, beta=10, 11 t-points, c64",
           "realizations_per_s": R / wall, "curves_per_s": len(jobs) / wall, "wall_s": wall,
           "matvec_Gtermamp_s": termamps / wall / 1e9, "failed": sum(1 for v in results.values() if v["status"]),
           "krylov_m": m or "library default", "ticks_per_sync": tps, "autotune": tune}
    # plain FP64 single-realisation path (complex128, one realisation at a time)
    nplain = 0 if args.batch_no_plain else min(8, R)
    t0 = time.perf_counter()
    diffs = []
    for r in range(nplain):
        N, q, J, h = reals[r]
        with syk.Terms(N, q, J, dtype="c128") as h64:
            for s in range(S):
                u, d = h64.random_state(1234 + r, s)
                nrm = torch.sqrt(torch.sum(torch.abs(u) ** 2) + torch.sum(torch.abs(d) ** 2))
                psi = torch.stack([u / nrm, d / nrm]).unsqueeze(0).contiguous()
                F64, _, _ = h64.otoc(N - 1, N - 2, beta, grid, psi=psi)
                diffs.append(np.max(np.abs(results[r * S + s]["F"] - F64[0])) / np.max(np.abs(F64[0])))
    plain_wall = time.perf_counter() - t0
    if nplain:
        out["plain_fp64_single_path"] = {"realizations_per_s": nplain / plain_wall, "realizations": nplain,
                                         "note": "syk_otoc complex128, one realisation and state at a time"}
    out["c64_vs_fp64_max_rel_F_diff"] = float(max(diffs)) if diffs else None
    for r in reals:
        r[3].close()
    return out


def otoc_served(args, syk, torch):
    """Served configuration (bounded): Poisson requests with N in 28..48
    weighted toward small N, k in {0.5,1,2,4}, beta in {2,5,10,20}; the arrival
    rate is set to ~75% of the capacity measured by a closed-loop pass.

    The mix is heavy-tailed (the work of a request grows like 2^(N/2) while its
    weight falls like 0.7^(N/2)), so a few hundred requests can carry much less
    or much more work per request than the served sample.  The closed-loop pass
    therefore measures capacity in work units per second (serve.work_estimate:
    terms x amplitudes x (grid points + sum |t|)), and the capacity in requests
    per second of the served sample is that rate over the served sample's mean
    work per request."""
    import numpy as np
    from paper_2311_00639_b300 import serve
    import syk_inputs as si

    kw = dict(t_max=args.serve_tmax, dt=args.serve_dt)
    n = args.serve_requests
    hbm = int(args.serve_hbm_gb * (1 << 30))

    def workload(count, seed):  # arrival times of a rate-1 Poisson process
        return [serve.Request(**r) for r in si.served_requests(count, rate=1.0, seed=seed, **kw)]

    # capacity: requests all present at t=0 (a separate sample of the same mix)
    cap_reqs = workload(args.serve_capacity_requests or n, 11)
    for r in cap_reqs:
        r.arrival = 0.0
    srv = serve.OtocServer(dtype="c64", max_slots=args.serve_slots, hbm_budget_bytes=hbm, ticks_per_step=8,
                           policy=args.serve_policy)
    t0 = time.perf_counter()
    res = srv.run(cap_reqs)
    cap_wall = time.perf_counter() - t0
    srv.close()
    reqs = workload(n, 12)
    rate, cap = serve.calibrated_rate(cap_reqs, cap_wall, reqs, args.serve_load)
    cap_work = sum(serve.work_estimate(r, None) for r in cap_reqs) / cap_wall
    mean_work = float(np.mean([serve.work_estimate(r, None) for r in reqs]))
    for r in reqs:
        r.arrival /= rate
    srv = serve.OtocServer(dtype="c64", max_slots=args.serve_slots, hbm_budget_bytes=hbm, ticks_per_step=8,
                           policy=args.serve_policy)
    t0 = time.perf_counter()
    res = srv.run(reqs)
    wall = time.perf_counter() - t0
    srv.close()
    summ = serve.summarize(res, wall, work={r.rid: serve.work_estimate(r, None) for r in reqs},
                           capacity_work_per_s=cap_work)
    summ.update({"arrival_rate_per_s": rate, "closed_loop_capacity_per_s": cap, "load": args.serve_load,
                 "capacity": {"requests": len(cap_reqs), "wall_s": cap_wall, "requests_per_s": len(cap_reqs) / cap_wall,
                              "work_units_per_s": cap_work,
                              "mean_work_per_request": sum(serve.work_estimate(r, None) for r in cap_reqs)
                              / len(cap_reqs)},
                 "served_mean_work_per_request": mean_work,
                 "workload": f"{n} Poisson requests, N 28..48 (P ~ 0.7^((N-28)/2)), k 0.5..4, beta 2..20, "
                             f"t 0..{args.serve_tmax:g} step {args.serve_dt:g}, c64, HBM budget "
                             f"{args.serve_hbm_gb:g} GiB, {args.serve_slots} slots, admission {args.serve_policy}; "
                             f"arrival rate = {args.serve_load:g} x closed-loop work rate / served mean work"})
    return summ


def paper_rows(args, syk, si, torch):
    """The paper's benchmark rows (supplement Sec. I.B: time per OTOC curve,
    one realisation, one state, t = 0..10 in 10 segments, sparse k = 3,
    beta = 0.05) through the single-realisation path syk_otoc, complex128 and
    complex64 (library Krylov defaults), one warm-up curve each."""
    import numpy as np

    grid = np.linspace(0.0, 10.0, 11)
    rows = []
    sizes = [(int(v), 3.0) for v in args.rows_N.split(",") if v]
    sizes += [(int(v), "dense") for v in args.rows_dense_N.split(",") if v]
    for N, k in sizes:
        q, J, _ = si.sample_dense_syk(N, seed=0) if k == "dense" else si.sample_sparse_syk(N, k, r=0)
        row = {"N": N, "k": k if k == "dense" else 3, "beta": 0.05, "terms": len(J)}
        for dtype in ("c128", "c64"):
            with syk.Terms(N, q, J, dtype=dtype) as h:
                h.otoc(N - 1, N - 2, 0.05, grid[:2], n_states=1, seed=9)  # warm-up (captures the Krylov loops)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                F, o, st = h.otoc(N - 1, N - 2, 0.05, grid, n_states=1, seed=9)
                row[f"{dtype}_s_per_curve"] = time.perf_counter() - t0
                row[f"{dtype}_matvecs"] = st.matvecs
                row[f"{dtype}_substeps"] = st.substeps
                row[f"{dtype}_otoc_t10"] = float(o[-1])
                if dtype == "c64":
                    row["c64_merged_terms"] = h.info["n_merged"]
        rows.append(row)
    return {"workload": "paper benchmark rows, sparse k=3 (and dense SYK with --rows-dense-N), beta=0.05, "
                        "one Philox state, 11 t-points",
            "rows": rows}


def config2(args, syk, si, torch):
    """The N=32 mixed-precision configuration: sparse SYK N=32, k=4
    (realisation r=0), Lanczos m=30, 64 Philox typical states (seed 7, ids
    0..63), t = 0..15 in steps of 0.1 (151 points), beta in {0, 5, 10}; every
    curve in complex64 states (FP64 scalars) and in complex128, both through
    the batched engine at the library's Krylov tolerances (1e-6 and 1e-12).  The complex64 error is stated against
    the complex128 curves for all 64 x 3 curves, and both are compared with
    the FP64 oracle's stored values (expm_multiply, states 0 and 1 at
    t in {0, 0.1, 1, 2.5, 5, 10, 15}; tests/golden/otoc_N32_k4_r0_typical.txt)."""
    import numpy as np

    N, S = 32, 64
    grid = np.round(np.arange(0.0, 15.0 + 1e-9, 0.1), 10)
    betas = (0.0, 5.0, 10.0)
    q, J, _ = si.sample_sparse_syk(N, 4.0, r=0)
    gold_rows = np.loadtxt(os.path.join(ROOT, "tests", "golden", "otoc_N32_k4_r0_typical.txt"), comments="#")
    curves, timing = {}, {}
    for dtype, tol in (("c64", None), ("c128", None)):
        with syk.Terms(N, q, J, dtype=dtype) as h, syk.Batch(dtype=dtype, max_slots=S * len(betas),
                                                             max_bytes=16 << 30, m=30, tol=tol) as b:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tag = 0
            keys = {}
            for beta in betas:
                for s in range(S):
                    assert b.submit(h, N - 1, N - 2, beta, grid, 7, s, tag)
                    keys[tag] = (beta, s)
                    tag += 1
            res = b.drain()
            timing[dtype] = {"s": time.perf_counter() - t0, "curves": len(res),
                             "matvecs": int(sum(r["matvecs"] for r in res)),
                             "failed": sum(1 for r in res if r["status"])}
            curves[dtype] = {keys[r["tag"]]: r["F"] for r in res}
    out = {"workload": f"N={N}, k=4, T={len(J)}, m=30, {S} Philox states, 151 t-points (0..15, step 0.1), "
                       "beta 0/5/10, batched engine", "timing": timing, "per_beta": {}}
    worst = 0.0
    for beta in betas:
        errs = [float(np.max(np.abs(curves["c64"][(beta, s)] - curves["c128"][(beta, s)])) /
                      np.max(np.abs(curves["c128"][(beta, s)]))) for s in range(S)]
        m64 = np.mean([curves["c64"][(beta, s)] for s in range(S)], axis=0)
        m128 = np.mean([curves["c128"][(beta, s)] for s in range(S)], axis=0)
        o64, o128 = m64.real / m64.real[0], m128.real / m128.real[0]
        r = gold_rows[gold_rows[:, 0] == beta]
        vs_oracle = {}
        for dtype in ("c64", "c128"):
            e = 0.0
            for s in (0, 1):
                rs = r[r[:, 1] == s]
                idx = [int(round(tv * 10)) for tv in rs[:, 2]]
                Fg = rs[:, 3] + 1j * rs[:, 4]
                e = max(e, float(np.max(np.abs(curves[dtype][(beta, s)][idx] - Fg)) / np.max(np.abs(Fg))))
            vs_oracle[dtype] = e
        out["per_beta"][f"{beta:g}"] = {"c64_vs_c128_max_rel_F": max(errs), "c64_vs_c128_median_rel_F": float(np.median(errs)),
                                        "otoc_mean_max_abs_diff": float(np.max(np.abs(o64 - o128))),
                                        "otoc_t15_c128": float(o128[-1]),
                                        "vs_fp64_oracle_subset": vs_oracle}
        worst = max(worst, max(errs), vs_oracle["c64"])
    out["c64_vs_fp64_max_rel_F"] = worst
    return out


# ------------------------------------------------------------- spin chains --
def oracle_spin_rows_rate(L, W, seconds=10.0, seed=77):
    """CPU oracle: sampled rows of H psi for the random-field Heisenberg chain
    from the definition (basis-state maps, numpy).  Returns (Gterm*amp/s,
    rows, T)."""
    import numpy as np

    import syk_inputs as si
    from oracle import spin

    x, z, h, _ = si.heisenberg_chain(L, W, r=0)
    rng = np.random.default_rng(seed)

    def run(nrows):
        rows = rng.integers(0, 1 << L, nrows).astype(np.uint64)
        needed = []
        spin.rows_of_Hpsi(L, x, z, h, rows, lambda g: needed.append(g.copy()) or np.zeros(len(g)))
        idx = np.unique(np.concatenate(needed))
        vals = si.philox_state(2 * L + 2, seed, 0, idx)  # inputs, generated outside the timed region
        t0 = time.perf_counter()
        spin.rows_of_Hpsi(L, x, z, h, rows, lambda g: vals[np.searchsorted(idx, g)])
        return time.perf_counter() - t0

    dt = run(256)
    nrows = int(min(1 << 20, max(256, 256 * seconds / max(dt, 1e-3))))
    dt = run(nrows)
    return len(h) * nrows / dt / 1e9, nrows, len(h)


def hpsi_rate(t, steps, warmup, torch, n_input=None):
    """Time `steps` H psi of handle t (block 0, one resident Philox state);
    the rate counts n_input terms per amplitude (default: the compiled strings)."""
    psi, _ = t.random_state(seed=1234, state_id=0, blocks=(0,))
    o = t.empty()
    dt = time_matvecs(t, psi, o, steps, warmup, torch)
    del psi, o
    torch.cuda.empty_cache()
    n = t.n_terms if n_input is None else n_input
    return {"Gtermamp_s": n * t.D * steps / dt / 1e9, "ms_per_Hpsi": dt * 1e3 / steps, "terms": n,
            "strings": t.n_terms, "passes": t.info["n_passes"], "tile_reads": t.info["n_tile_reads"], "steps": steps}


def outlook_hpsi(args, syk, si, torch):
    """Informational keys of the benchmark line: H psi of the outlook's two
    models at the benchmark's scale (complex64, 2^31 amplitudes): the
    random-field Heisenberg chain (L=31, W=5, 124 strings) and the N=64, k=4
    quadruples with complex couplings J + iM (M ~ 0.1 J, 522 strings).  A
    failure here is recorded in place of the numbers and never stops the line."""
    import numpy as np

    out = {}
    steps = max(1, min(5, args.steps))
    try:
        x, z, h, _ = si.heisenberg_chain(31, 5.0, r=0)
        with syk.PauliTerms(31, x, z, h, dtype="c64") as t:
            out["spin_chain_L31"] = hpsi_rate(t, steps, 2, torch)
    except Exception as e:  # informational only
        out["spin_chain_L31"] = {"error": str(e)[:300]}
    try:
        q, J, _ = si.sample_sparse_syk(64, 4.0, r=0)
        M = 0.1 * np.random.default_rng(900).normal(size=len(J)) * math.sqrt(float(np.mean(J ** 2)))
        q, J, M, relabel = locality_terms_complex(syk, 64, q, J, M, args)
        with syk.Terms.complex(64, q, J, M, dtype="c64") as t:
            out["nonhermitian_N64"] = dict(hpsi_rate(t, steps, 2, torch, n_input=len(J)), relabelled=bool(relabel))
    except Exception as e:  # informational only
        out["nonhermitian_N64"] = {"error": str(e)[:300]}
    return out


def spin_leg(args, syk, si, torch):
    """The outlook's spin chains: the random-field Heisenberg chain
    H = sum S_i.S_{i+1} - sum h_i S^z_i (periodic, W = 5) as Pauli strings.
    H psi at L = spin_L (complex64 and complex128, inputs resident), and
    OTOC curves (W = Z_0, V = Z_{L/2}, beta = spin_beta (infinite temperature
    by default), t = 0..10 in 10 segments, one Philox state) at
    L = spin_otoc_L.  At finite beta the raw F grows like e^{beta |E_min|}
    (an extensive energy), so the chain is shifted by an identity string of
    weight S/2, S = sum |h| (E_min lies in [-S, 0] since Tr H = 0): F scales
    by e^{-beta S/2}, the OTOC ratio is unchanged, and complex64 weights stay
    within e^{+-beta S/2} (in float32 range while beta S/2 < ~80)."""
    import numpy as np

    Wd = 5.0
    L = args.spin_L
    x, z, h, _ = si.heisenberg_chain(L, Wd, r=0)
    out = {"workload": f"random-field Heisenberg chain, L={L}, W={Wd:g}, periodic, D=2^{L}"}
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    for dtype, steps in (("c64", args.steps), ("c128", max(1, min(3, args.steps)))):
        with syk.PauliTerms(L, x, z, h, dtype=dtype) as t:
            if dtype == "c64":
                clocks.start()
            out[dtype] = hpsi_rate(t, steps, args.warmup if dtype == "c64" else 1, torch)
            if dtype == "c64":
                out["clocks"] = clocks.stop()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    peak_slots = props.multi_processor_count * 128 * sm_max * 1e6 / 1e12
    ms = out["c64"]["ms_per_Hpsi"]
    T, D = out["c64"]["terms"], 1 << L
    out["roofline_c64"] = {"bound": "alu", "achieved": ISSUE_SLOTS_PER_TERM_AMP * T * D / (ms / 1e3) / 1e12,
                           "peak": peak_slots, "unit": "Tslot/s",
                           "frac": ISSUE_SLOTS_PER_TERM_AMP * T * D / (ms / 1e3) / 1e12 / peak_slots,
                           "hbm_gbs_achieved": 2 * D * 8 / (ms / 1e3) / 1e9,
                           "hbm_peak_gbs": peaks.get("hbm_gbs", 6400.0), "algorithmic_bytes": 2 * D * 8}
    # OTOC curves
    Lo = args.spin_otoc_L
    beta = args.spin_beta
    xo, zo, ho, _ = si.heisenberg_chain(Lo, Wd, r=1)
    if beta > 0:
        shift = 0.5 * float(np.sum(np.abs(ho)))
        xo, zo, ho = np.append(xo, 0), np.append(zo, 0), np.append(ho, shift)
    Wm, Vm = si.pauli_mask({0: "Z"}), si.pauli_mask({Lo // 2: "Z"})
    grid = np.linspace(0.0, 10.0, 11)
    curves = {}
    for dtype in ("c64", "c128"):
        with syk.PauliTerms(Lo, xo, zo, ho, dtype=dtype) as t:
            t.pauli_otoc(Wm, Vm, beta, grid[:2], n_states=1, seed=5)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            F, o, st = t.pauli_otoc(Wm, Vm, beta, grid, n_states=1, seed=5)
            wall = time.perf_counter() - t0
            curves[dtype] = {"s_per_curve": wall, "matvecs": st.matvecs, "otoc": list(o), "F": F[0]}
    diff = float(np.max(np.abs(curves["c64"]["F"] - curves["c128"]["F"])) / np.max(np.abs(curves["c128"]["F"])))
    for c in curves.values():
        c.pop("F")
    out["otoc"] = {"workload": f"L={Lo}, W={Wd:g}, W=Z_0, V=Z_{Lo // 2}, beta={beta:g}, t=0..10 (11 points), "
                               "one Philox state, Lanczos defaults (m=20 c64, m=30 c128)"
                               + (", H shifted by sum|h|/2" if beta > 0 else ""),
                   **curves, "c64_vs_c128_max_rel_F_diff": diff}
    if not args.no_cpu:
        v, nrows, Tc = oracle_spin_rows_rate(L, Wd)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"{nrows} random rows of H psi (L={L}, T={Tc}) from the definition"}
    return out


# --------------------------------------------------------- non-Hermitian ----
def nonherm_leg(args, syk, si, torch):
    """Non-Hermitian sparse SYK (couplings J + iM, M Gaussian with 0.1 the
    spread of J: weakly non-Hermitian, so that the raw F, which grows like
    e^{4 t max Im lambda}, stays readable): H psi at N = args.N (complex64,
    inputs resident; every term is a real-class and an imaginary-class
    string) and infinite-temperature OTOC curves (W(t) = e^{iH^dag t} W e^{-iHt},
    a = N-1, b = N-2, t = 0..10 in 10 segments, one Philox state, Arnoldi) at
    N = 30, k = 3."""
    import numpy as np

    def couplings(N, k, r):
        q, J, _ = si.sample_sparse_syk(N, k, r=r)
        M = 0.1 * np.random.default_rng(900 + r).normal(size=len(J)) * math.sqrt(float(np.mean(J ** 2)))
        return q, J, M

    q, J, M = couplings(args.N, args.k, 0)
    q, J, M, relabel = locality_terms_complex(syk, args.N, q, J, M, args)
    out = {"workload": f"non-Hermitian sparse SYK N={args.N}, k={args.k:g}, couplings J + iM (M ~ 0.1 J), "
                       "one parity block" + (", Majoranas relabelled for locality" if relabel else ""),
           "relabel": relabel}
    with syk.Terms.complex(args.N, q, J, M, dtype="c64") as h:
        out["Hpsi_c64"] = dict(hpsi_rate(h, args.steps, args.warmup, torch, n_input=len(J)),
                               note="rate counts input terms (quads); each compiles to two strings")
    if args.no_otoc:
        return out
    grid = np.linspace(0.0, 10.0, 11)
    q, J, M = couplings(30, 3.0, 1)
    curves = {}
    for dtype in ("c64", "c128"):
        with syk.Terms.complex(30, q, J, M, dtype=dtype) as h:
            h.otoc_nonhermitian(29, 28, grid[:2], n_states=1, seed=5)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            F, o, st = h.otoc_nonhermitian(29, 28, grid, n_states=1, seed=5)
            curves[dtype] = {"s_per_curve": time.perf_counter() - t0, "matvecs": st.matvecs,
                             "substeps": st.substeps, "otoc": list(o), "F": F[0]}
    diff = float(np.max(np.abs(curves["c64"]["F"] - curves["c128"]["F"])) / np.max(np.abs(curves["c128"]["F"])))
    for c in curves.values():
        c.pop("F")
    out["otoc"] = {"workload": "N=30, k=3, couplings J + iM (M ~ 0.1 J), a=29, b=28, beta=0, t=0..10 (11 points), one Philox "
                               "state, Arnoldi (m=20 c64, m=30 c128)", **curves, "c64_vs_c128_max_rel_F_diff": diff}
    return out


# ------------------------------------------------------------------ ours ----
def build_lib():
    spec = importlib.util.spec_from_file_location("_syk_build", os.path.join(ROOT, "paper_2311_00639_b300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()


def max_over_ranks(v, dist, device="cuda"):
    """The maximum of a per-rank float over all ranks (a replica job takes as
    long as its slowest rank); v itself without a process group."""
    if dist is None:
        return v
    import torch

    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def replica_terms(si, N, k, rank):
    """Replicas only: rank r runs disorder realisation r of the workload."""
    q, J, _ = si.sample_sparse_syk(N, k, r=rank)
    return q, J


def time_matvecs(h, psi, out, steps, warmup, torch):
    for _ in range(warmup):
        h.apply_H(psi, 0, out=out)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        h.apply_H(psi, 0, out=out)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def ours(args):
    import numpy as np
    import torch

    build_lib()
    import paper_2311_00639_b300 as syk
    import syk_inputs as si

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    barrier = (lambda: dist.barrier()) if dist else (lambda: None)

    if args.dense:  # every quadruple (the relabelling search is for sparse term lists)
        args.no_relabel = True
        q0, J0, _ = si.sample_dense_syk(args.N, seed=rank)
    else:
        q0, J0 = replica_terms(si, args.N, args.k, rank)
    q, J, relabel_info = locality_terms(syk, args.N, q0, J0, args)
    h = syk.Terms(args.N, q, J, dtype="c64")
    T, D = h.n_terms, h.D
    psi, _ = h.random_state(seed=1234, state_id=rank, blocks=(0,))
    out = h.empty()
    props = torch.cuda.get_device_properties(local)

    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    dt = time_matvecs(h, psi, out, args.steps, args.warmup, torch)
    clk = clocks.stop()
    barrier()
    dt = max_over_ranks(dt, dist)
    per_step = dt / args.steps
    value = world * T * D * args.steps / dt / 1e9

    # the same step with the identity Jordan-Wigner order (for comparison)
    identity = None
    if relabel_info is not None and not args.no_identity:
        h0 = syk.Terms(args.N, q0, J0, dtype="c64")
        k0 = max(3, min(5, args.steps))
        d0 = max_over_ranks(time_matvecs(h0, psi, out, k0, 2, torch), dist)
        identity = {"value": world * T * D * k0 / d0 / 1e9, "unit": UNIT, "ms_per_step": d0 * 1e3 / k0,
                    "passes": h0.info["n_passes"], "tile_reads": h0.info["n_tile_reads"],
                    "note": "identity Jordan-Wigner order, same couplings (not the timed value)"}
        h0.close()
        relabel_info.update({"passes": h.info["n_passes"], "tile_reads": h.info["n_tile_reads"]})

    # e2e through the public API: every step copies its input psi from pinned
    # host memory to the device, applies H (syk_apply_H) and copies the result
    # back to pinned host memory.  Steps are pipelined as a streaming caller
    # would run them: three streams (host->device, compute, device->host) and
    # two device buffer sets, so step i+1's upload and step i's download (the
    # two directions of the host link) overlap step i's H psi; events keep
    # every buffer from being overwritten while it is still read.  The timed
    # region spans the first upload to the last download.
    e2e = None
    if not args.no_e2e:
        ke = max(4, min(8, args.steps))
        hpsi = torch.empty(D, dtype=torch.complex64, pin_memory=True)
        hout = torch.empty(D, dtype=torch.complex64, pin_memory=True)
        hpsi.copy_(psi)
        din, dout = [psi, torch.empty_like(psi)], [out, torch.empty_like(out)]
        s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_cmp = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]

        def e2e_steps(n):
            for i in range(n):
                b = i % 2
                if i >= 2:
                    s_in.wait_event(ev_cmp[b])  # step i-2 has finished reading din[b]
                with torch.cuda.stream(s_in):
                    din[b].copy_(hpsi, non_blocking=True)
                ev_in[b].record(s_in)
                s_cmp.wait_event(ev_in[b])
                if i >= 2:
                    s_cmp.wait_event(ev_out[b])  # step i-2's result has left dout[b]
                h.apply_H(din[b], 0, out=dout[b], stream=s_cmp)
                ev_cmp[b].record(s_cmp)
                s_out.wait_event(ev_cmp[b])
                with torch.cuda.stream(s_out):
                    hout.copy_(dout[b], non_blocking=True)
                ev_out[b].record(s_out)

        e2e_steps(2)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_steps(ke)
        torch.cuda.synchronize()
        de = max_over_ranks((time.perf_counter() - t0) / ke, dist)
        e2e = {"value": world * T * D / de / 1e9, "unit": UNIT, "h2d_bytes_per_step": D * 8,
               "d2h_bytes_per_step": D * 8, "ms_per_step": de * 1e3, "steps": ke,
               "pipeline": "3 streams, 2 device buffer sets: upload i+1 and download i overlap H psi i"}

        # The host link alone: one step's upload, its download, and both at
        # once on their two streams (the pipelined e2e step cannot beat the
        # slower of the two-direction copy and the H psi).
        def copies(h2d, d2h, reps=2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                if h2d:
                    with torch.cuda.stream(s_in):
                        din[0].copy_(hpsi, non_blocking=True)
                if d2h:
                    with torch.cuda.stream(s_out):
                        hout.copy_(dout[1], non_blocking=True)
            torch.cuda.synchronize()
            return (time.perf_counter() - t0) / reps

        th, td, tb = copies(True, False), copies(False, True), copies(True, True)
        bound = max(tb, per_step)
        e2e["host_link"] = {"h2d_GBps": D * 8 / th / 1e9, "d2h_GBps": D * 8 / td / 1e9,
                            "both_directions_ms": tb * 1e3, "step_bound_ms": bound * 1e3,
                            "frac_of_bound": bound / de,
                            "note": "bound = max(upload and download together, H psi); frac = bound / e2e step"}
        del hpsi, hout, din, dout
        torch.cuda.empty_cache()

    # float64 states (complex128)
    fp64 = None
    if not args.no_fp64:
        del out
        psi64 = None
        h64 = syk.Terms(args.N, q, J, dtype="c128")
        psi64, _ = h64.random_state(seed=1234, state_id=rank, blocks=(0,))
        out64 = h64.empty()
        k64 = max(1, min(3, args.steps))
        d64 = max_over_ranks(time_matvecs(h64, psi64, out64, k64, min(args.warmup, 2), torch), dist)
        fp64 = {"value": world * T * D * k64 / d64 / 1e9, "unit": UNIT, "ms_per_step": d64 * 1e3 / k64,
                "dtype": "c128 (f64)"}
        # FP64 roofline: a complex128 amplitude times a real (or imaginary) coefficient is
        # 2 DFMA = 4 FLOP per term x amplitude, against the DFMA rate measured now
        try:
            dfma = syk.probe_fp64()
            ach = 4.0 * T * D * k64 / d64 / 1e12
            fp64["roofline"] = {"bound": "alu", "achieved": ach, "peak": 2.0 * dfma / 1e12, "unit": "TFLOP/s (FP64)",
                                "frac": ach / (2.0 * dfma / 1e12),
                                "peak_source": "syk_probe_fp64: independent DFMA chains on all SMs, measured in "
                                               "this run (2 FLOP per DFMA)"}
        except Exception as e:  # informational
            fp64["roofline"] = {"error": str(e)[:200]}
        del psi64, out64
        h64.close()

    # the same kernel on an L2-resident block (N=46: 32 MiB per vector, input +
    # output 64 MiB of the 126 MB L2, one pass, 2048 tiles), with one term per
    # input tile (quads of a k=8 sample kept only while their compiled flip
    # mask reads a tile no earlier kept term reads): its rate of staging 16 KiB
    # input tiles from L2 into shared memory is the ceiling of the N=64 kernel,
    # which stages one tile per run of terms that read it
    l2res = None
    if not args.no_l2:
        import numpy as np

        q46, J46, _ = si.sample_sparse_syk(46, 8.0, r=rank)
        keep, seen = [], set()
        for i in range(len(J46)):
            xi = int(syk.compile_terms_host(46, q46[i:i + 1], J46[i:i + 1])["x"][0]) >> 11
            if xi not in seen:
                seen.add(xi)
                keep.append(i)
        q46, J46 = np.asarray(q46)[keep], np.asarray(J46)[keep]
        h46 = syk.Terms(46, q46, J46, dtype="c64")
        h46.replan(256 << 20, 0.0)
        p46, _ = h46.random_state(seed=7, state_id=0, blocks=(0,))
        o46 = h46.empty()
        k46 = 100
        d46 = time_matvecs(h46, p46, o46, k46, 10, torch)
        rate = h46.n_terms * h46.D * k46 / d46
        l2res = {"N": 46, "terms": h46.n_terms, "D": h46.D, "value": rate / 1e9, "unit": UNIT,
                 "sample": "k=8 quads with distinct input tiles (one term per staged tile)",
                 "tile_reads": h46.info["n_tile_reads"],
                 "staged_GBps": h46.info["n_tile_reads"] * h46.D * 8 * k46 / d46 / 1e9}
        h46.close()
        del p46, o46

    # roofline of the matvec kernel
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6400.0)
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    peak_slots = props.multi_processor_count * 128 * sm_max * 1e6 / 1e12  # Tslot/s
    achieved_slots = ISSUE_SLOTS_PER_TERM_AMP * T * D / per_step / 1e12
    t_bytes = 2 * D * 8 / (hbm * 1e9)
    t_alu = ISSUE_SLOTS_PER_TERM_AMP * T * D / (peak_slots * 1e12)
    staged_gbps = h.info["n_tile_reads"] * D * 8 / per_step / 1e9  # L2 -> shared memory input staging
    roof = {"bound": "alu" if t_alu >= t_bytes else "hbm", "achieved": achieved_slots, "peak": peak_slots,
            "unit": "Tslot/s", "frac": achieved_slots / peak_slots, "traffic": None,
            "peak_source": f"{props.multi_processor_count} SMs x 128 lanes x {sm_max:.0f} MHz (measured max clock)",
            "algorithmic_bytes": 2 * D * 8, "hbm_time_ms": t_bytes * 1e3, "alu_time_ms": t_alu * 1e3,
            "hbm_gbs_achieved": 2 * D * 8 / per_step / 1e9, "hbm_peak_gbs": hbm,
            "tile_reads": h.info["n_tile_reads"], "staged_GBps": staged_gbps,
            "l2_resident_ceiling": l2res,
            "frac_of_l2_resident": staged_gbps / l2res["staged_GBps"] if l2res else None}
    roof["traffic"] = measured_traffic(syk, args.N, q, J)
    # The binding limit of this kernel: every term x amplitude needs its own
    # 8-byte input from L2 (terms of a pass that read the same tile share one
    # staged copy), so the L2 -> shared-memory staging rate bounds it.  Staged
    # bytes per H psi: the pass runs' input tiles plus one partial-sum tile per
    # output tile in every pass after the first.  The peak is the same pipeline
    # shape with no arithmetic (syk_probe_staging, consumers reading each tile
    # once), measured now on a 32 MiB L2-resident buffer.
    try:
        pb = torch.empty(32 << 20, dtype=torch.uint8, device="cuda")
        pb.random_()
        stage_peak = syk.probe_staging(pb, 1, 8192) / 1e12
        stage_peak0 = syk.probe_staging(pb, 0, 8192) / 1e12
        ldg_peak = syk.probe_staging(pb, -1, 8192) / 1e12
        del pb
        staged = (h.info["n_tile_reads"] + h.info["n_passes"] - 1) * D * 8
        roof_l2 = {"bound": "l2", "achieved": staged / per_step / 1e12, "peak": stage_peak, "unit": "TB/s",
                   "frac": staged / per_step / 1e12 / stage_peak, "staged_bytes_per_step": staged,
                   "peak_source": "syk_probe_staging: 16 KiB bulk copies of a 32 MiB L2-resident buffer into "
                                  "the shared-memory stages and CTAs per SM of the store passes, consumers read each tile once; "
                                  "measured in this run",
                   "probe_TBps": {"staging_no_reads": stage_peak0, "staging_one_read": stage_peak,
                                  "plain_global_loads": ldg_peak},
                   "time_bound_ms": staged / (stage_peak * 1e12) * 1e3,
                   "alu_frac_ceiling": t_alu / (staged / (stage_peak * 1e12))}
    except Exception as e:  # informational
        roof_l2 = {"error": str(e)[:200]}
    # The second data path of the kernel: the consumers read every staged
    # input once per term of its run (8 bytes per term x amplitude) and, in
    # every pass after the first, the partial-sum tile once, with 16-byte
    # shared-memory loads.  Peak: the same loads with nothing else running
    # (syk_probe_smem), measured now.
    try:
        lds_peak = syk.probe_smem() / 1e12
        lds = (T + h.info["n_passes"] - 1) * D * 8
        roof_smem = {"bound": "smem", "achieved": lds / per_step / 1e12, "peak": lds_peak, "unit": "TB/s",
                     "frac": lds / per_step / 1e12 / lds_peak, "lds_bytes_per_step": lds,
                     "peak_source": "syk_probe_smem: 16-byte shared-memory loads, 8 CTAs of 128 threads per SM, "
                                    "measured in this run",
                     "time_bound_ms": lds / (lds_peak * 1e12) * 1e3,
                     "alu_frac_ceiling": t_alu / (lds / (lds_peak * 1e12))}
    except Exception as e:  # informational
        roof_smem = {"error": str(e)[:200]}

    outlook = None
    if rank == 0 and not args.no_outlook:
        outlook = outlook_hpsi(args, syk, si, torch)

    batched = served = None
    if not args.no_otoc:
        torch.cuda.empty_cache()
        batched = otoc_batched(args, syk, si, torch, rank)
        if rank == 0:
            served = otoc_served(args, syk, torch)

    cpu = None
    if rank == 0 and not args.no_cpu:
        v, nrows, _, cores, calls = cpp_rows_rate(args.N, args.k, seconds=10.0)
        vn, nrows_np, _, _ = oracle_rows_rate(args.N, args.k, seconds=4.0)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"output rows [0, {nrows}) of H_UU psi (N={args.N}, T={T}), C++/OpenMP FP64 baseline "
                         f"(oracle/cpu_baseline.cpp), {calls} calls in about 10 s",
               **host_info(), "full_block_hpsi": cpp_full_rates(args.k),
               "numpy_oracle_rows": {"value": vn, "unit": UNIT, "cores": 1,
                                     "sample": f"{nrows_np} random rows from the definition (basis-state maps)"}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c64 (f32 states)", "data": "synthetic",
                "config": {**workload_config(args, T), "parallelism": f"replicas x{world}",
                           "matvec_passes": h.info["n_passes"], "relabel": relabel_info},
                "jw_identity_order": identity,
                "gpu_launches": args.steps * h.info["n_passes"], "roofline": roof, "roofline_l2_staging": roof_l2,
                "roofline_smem": roof_smem,
                "cpu_baseline": cpu, "e2e": e2e,
                "fp64": fp64, "clocks": clk, "gpu": props.name, "otoc_batched": batched, "otoc_served": served,
                "outlook_hpsi": outlook}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def otoc_only(args):
    import torch

    build_lib()
    import paper_2311_00639_b300 as syk
    import syk_inputs as si

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if args.mode == "n64-otoc":
        # End-to-end OTOC at N=64: complex64 states, FP64 scalars, Lanczos with a stored
        # basis of m+1 = 11 vectors (4 + 11 vectors of 16 GiB live; --n64-two-pass keeps 3
        # by regenerating the basis), beta=10, one Philox state, t in {0, 0.5}; both blocks.
        q, J, _ = si.sample_sparse_syk(args.N, args.k, r=0)
        q, J, _ = locality_terms(syk, args.N, q, J, args)  # keeps Majoranas N-1, N-2 (the OTOC's) in place
        h = syk.Terms(args.N, q, J, dtype="c64")
        grid = [0.0, 0.5]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        two_pass = args.n64_two_pass
        F, o, st = h.otoc(args.N - 1, args.N - 2, 10.0, grid, n_states=1, seed=2024, m=args.n64_m,
                          two_pass=two_pass)
        wall = time.perf_counter() - t0
        line = {"metric": "end-to-end OTOC time per t-point at N=64 (c64 states, FP64 scalars)",
                "value": wall / len(grid), "unit": "s/point", "higher_is_better": False,
                "config": {"workload": f"N={args.N}, k={args.k:g}, T={h.n_terms}, beta=10, 1 state, t={grid}, "
                                       f"Lanczos m={args.n64_m} {'two-pass' if two_pass else 'stored basis'}",
                           "wall_s": wall, "matvecs": st.matvecs,
                           "substeps": st.substeps, "F": [[z.real, z.imag] for z in F[0]], "otoc": list(o),
                           "s_per_matvec": wall / max(1, st.matvecs)}}
        print(json.dumps(line), flush=True)
        return
    if args.mode == "paper-rows":
        res = paper_rows(args, syk, si, torch)
        line = {"metric": "time per OTOC curve (the paper's benchmark rows: one realisation, one state, "
                          "t = 0..10 in 10 segments)", "value": res["rows"][0]["c128_s_per_curve"], "unit": "s",
                "higher_is_better": False, "config": res}
        print(json.dumps(line), flush=True)
        return
    if args.mode == "config2":
        res = config2(args, syk, si, torch)
        line = {"metric": "complex64 OTOC error vs FP64 (N=32, 64 states, 151 points, beta 0/5/10)",
                "value": res["c64_vs_fp64_max_rel_F"], "unit": "max |dF| / max |F|", "higher_is_better": False,
                "config": res}
        print(json.dumps(line), flush=True)
        return
    if args.mode == "spin":
        res = spin_leg(args, syk, si, torch)
        line = {"metric": "spin-chain H·ψ Gterm·amp/s (random-field Heisenberg, complex64)",
                "value": res["c64"]["Gtermamp_s"], "unit": UNIT, "higher_is_better": True, "steps": args.steps,
                "warmup": args.warmup, "dtype": "c64 (f32 states)", "data": "synthetic", "config": res}
        print(json.dumps(line), flush=True)
        return
    if args.mode == "nonherm":
        res = nonherm_leg(args, syk, si, torch)
        line = {"metric": "non-Hermitian SYK H·ψ Gterm·amp/s (complex64) and Arnoldi OTOC curves",
                "value": res["Hpsi_c64"]["Gtermamp_s"], "unit": UNIT, "higher_is_better": True,
                "steps": args.steps, "warmup": args.warmup, "dtype": "c64 (f32 states)", "data": "synthetic",
                "config": res}
        print(json.dumps(line), flush=True)
        return
    if args.mode == "otoc-batch":
        res = otoc_batched(args, syk, si, torch)
        line = {"metric": "OTOC realizations/s (batched)", "value": res["realizations_per_s"],
                "unit": "realizations/s", "higher_is_better": True, "config": res}
    else:
        res = otoc_served(args, syk, torch)
        line = {"metric": "OTOC served p50/p99 latency", "value": res["p50_latency_s"], "unit": "s",
                "higher_is_better": False, "config": res}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "ours" and args.mode != "all":
        otoc_only(args)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
