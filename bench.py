"""Benchmark: f + grad evaluations per second of Alg. 2 (fg_implicit) on one GB300.

Workload (one "step" = one full evaluation, the fused pass over V plus the model terms):
    n = 256 features, d = 4, r = 16, p = 2^24 Gaussian-mixture samples (16 unit-norm means,
    Dirichlet(1) weights, sigma = 0.1), nu = 1/p, V stored in BF16 (8.6 GB, far larger than
    L2, so no flush is needed between steps). The same samples in FP32 are timed beside it.

Prints ONE JSON line (rank 0). `--impl reference` times the FP64 CPU oracle on the host cores
instead, on a bounded sample of the same workload.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_FEAT, D, R, P_FULL, SIGMA, N_MEANS, SEED = 256, 4, 16, 1 << 24, 0.1, 16, 2024
WORKLOAD = "gmm_n256_d4_r16_p16777216"


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        pk = json.load(open(path))
        return dict(hbm_gbs=pk["hbm_gbs"], sm_max_mhz=pk.get("sm_max_mhz", 2070.0), src="measured")
    return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, src="fallback")


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


class UtilSampler:
    """nvidia-smi utilization.gpu (percent of the sample period in which a kernel ran) sampled
    every 100 ms while the block runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.values = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=utilization.gpu",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            try:
                self.values.append(float(line.strip()))
            except ValueError:
                pass

    def mean(self):
        return statistics.mean(self.values) if self.values else None


def strip_comments(src):
    """C/C++/CUDA source without its comments and blank lines (string and character literals
    kept as they are), so that a comment-only edit leaves the code hash unchanged."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    lines = (line.rstrip() for line in "".join(out).splitlines())
    return "\n".join(line for line in lines if line)


def kernel_source_hash(files=("fg_tc.cu", "tc_common.cuh")):
    """Hash of a fused pass's code (comments excluded)."""
    h = hashlib.sha256()
    for f in files:
        p = os.path.join(ROOT, "paper_1911_03813_gb300", "csrc", f)
        if os.path.exists(p):
            h.update(strip_comments(open(p, encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_tag):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        t = json.load(open(path)).get(kernel_tag)
    except ValueError:
        return None
    files = tuple(t.get("sources", ("fg_tc.cu", "tc_common.cuh"))) if t else ()
    if not t or t.get("source_hash") != kernel_source_hash(files):
        return None
    return t.get("dram_bytes_per_launch_full")


def cpu_baseline(dev, seconds=12.0, p_sample=1 << 17):
    """The FP64 oracle (NumPy, host BLAS threads) on a bounded sample of the workload, scaled to
    full-workload evaluations per second. Beside it, the GPU's f, g_lambda and G_A on the same
    sample in each storage type against the oracle: on the stored (rounded) values, which is
    the error of the GPU arithmetic, and on the FP64 samples, which adds the rounding of V."""
    import numpy as np
    import torch

    import oracle
    from oracle import formats
    from paper_1911_03813_gb300 import inputs, stmf
    data = inputs.gmm(N_FEAT, p_sample, N_MEANS, SIGMA, seed=SEED)
    Vt = np.ascontiguousarray(data["V"].T)
    lam, A = inputs.random_model(N_FEAT, R, seed=SEED + 1)
    ref64 = oracle.fg_implicit(None, Vt, lam, A, D)

    def rel(a, b):
        return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))

    accuracy = {}
    lam_t = torch.tensor(lam, device=dev)
    A_t = torch.tensor(np.ascontiguousarray(A.T), device=dev).T
    for dt in ("bf16", "f32", "e4m3"):
        st = inputs.to_storage(data["V"], dt, device=dev)
        f, gl, GA = stmf.fg(st, None, D, lam_t, A_t)
        got = (f.item(), gl.cpu().numpy(), GA.cpu().numpy())
        bits = inputs.storage_bits(st)
        stored = (formats.decode_bf16(bits) if dt == "bf16" else
                  formats.dequantize_e4m3(bits, st["scale"].cpu().numpy()) if dt == "e4m3" else
                  np.asarray(bits, dtype=np.float64))
        ref = oracle.fg_implicit(None, np.ascontiguousarray(stored.T), lam, A, D)
        accuracy[dt] = {
            "vs_oracle_on_stored_values": {"f": abs(got[0] - ref[0]) / abs(ref[0]),
                                           "g_lambda": rel(got[1], ref[1]),
                                           "G_A": rel(got[2], ref[2])},
            "vs_oracle_on_fp64_samples": {"f": abs(got[0] - ref64[0]) / abs(ref64[0]),
                                          "g_lambda": rel(got[1], ref64[1]),
                                          "G_A": rel(got[2], ref64[2])}}
        del st
    k, el = oracle_time(Vt, lam, A, seconds)
    per_eval_full = el / k * (P_FULL / p_sample)
    cores = len(os.sched_getaffinity(0))
    one = one_core_oracle(p_sample, seconds / 2)
    return dict(value=1.0 / per_eval_full, unit="evals/s", cores=cores, kind="oracle",
                sample="%d of %d samples (n=%d, d=%d, r=%d), %d evaluations in %.1f s, scaled "
                       "by p" % (p_sample, P_FULL, N_FEAT, D, R, k, el),
                one_core=one, accuracy=accuracy)


def oracle_time(Vt, lam, A, seconds):
    """(evaluations, seconds) of the FP64 oracle repeated for about `seconds`."""
    import oracle
    t0 = time.perf_counter()
    k = 0
    while True:
        oracle.fg_implicit(None, Vt, lam, A, D)
        k += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            return k, el


def one_core_oracle(p_sample, seconds):
    """The same oracle timing in a fresh process restricted to one core (affinity and every BLAS
    thread count set to 1 before NumPy loads), scaled to the whole workload like the all-core
    figure."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
              "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    try:
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-one-core",
                              str(p_sample), str(seconds)], env=env, capture_output=True,
                             text=True, timeout=600)
        res = json.loads(out.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError) as e:
        return {"error": str(e)[:200]}
    per_full = res["seconds"] / res["evals"] * (P_FULL / p_sample)
    return {"value": 1.0 / per_full, "unit": "evals/s", "cores": 1,
            "sample": "%d of %d samples, %d evaluations in %.1f s on one core, scaled by p"
                      % (p_sample, P_FULL, res["evals"], res["seconds"])}


def oracle_one_core_main(p_sample, seconds):
    os.sched_setaffinity(0, {sorted(os.sched_getaffinity(0))[0]})
    import numpy as np

    from paper_1911_03813_gb300 import inputs
    data = inputs.gmm(N_FEAT, p_sample, N_MEANS, SIGMA, seed=SEED)
    Vt = np.ascontiguousarray(data["V"].T)
    lam, A = inputs.random_model(N_FEAT, R, seed=SEED + 1)
    k, el = oracle_time(Vt, lam, A, seconds)
    print(json.dumps({"evals": k, "seconds": el}), flush=True)


def make_requests(count, seed, dev, pool=256):
    """Serving requests: n, p log-uniform in [8, 128] x [1e3, 1e6], d in {3, 4}, r in [1, 16],
    sigma log-uniform in [1e-4, 1e-1], four seeded starts each. The samples come from a pool of
    `pool` seeded Gaussian-mixture sets in pinned host memory (BF16; generated on the device and
    copied once before the clock starts), request k taking set k % pool: 4096 distinct sets of
    this size would hold about 50 GB of pinned host memory. Each request still carries its own
    d, r and starts, and the server copies its samples to the device at admission."""
    import numpy as np
    import torch

    from paper_1911_03813_gb300 import inputs
    g = np.random.default_rng(seed)
    sets = []
    for k in range(min(count, pool)):
        n = int(round(np.exp(g.uniform(np.log(8), np.log(128)))))
        p = int(round(np.exp(g.uniform(np.log(1e3), np.log(1e6)))))
        sigma = float(np.exp(g.uniform(np.log(1e-4), np.log(1e-1))))
        st = inputs.gmm_device(n, p, 16, sigma, seed * 100003 + k, dev, out_dtype="bf16")
        host = torch.empty(st["data"].shape, dtype=torch.int16, pin_memory=True)
        host.copy_(st["data"].view(torch.int16))
        sets.append(dict(V=dict(data=host.numpy(), n=n, dtype="bf16"), n=n, p=p, keep=host))
        del st
    out = []
    for k in range(count):
        s_ = sets[k % len(sets)]
        n = s_["n"]
        d = int(g.integers(3, 5))
        r = int(g.integers(1, 17))
        x0 = []
        for s in range(4):
            lam0, A0 = inputs.random_model(n, r, seed=seed * 7919 + 4 * k + s, lam="equal")
            x0.append(np.concatenate([lam0, A0.reshape(-1, order="F")]))
        out.append(dict(V=s_["V"], x0=np.array(x0), d=d, n_=n, p=s_["p"], r=r, keep=s_["keep"]))
    return out


def serving_bench(n_requests, seed, dev, device_index, sweep=(), fixed_rate=80.0):
    """Continuous batching through stmf_server_*: a saturated run fixes the capacity, then Poisson
    arrivals at 0.8x that rate give the latency percentiles; `sweep` lists further multiples of
    the saturated rate, each run on the same requests with its own arrival draw. A last run
    offers a quarter of the requests at a fixed rate (`fixed_rate` requests/s, 4 fits each), so
    the latency can be compared at the same load across versions whose capacity differs."""
    import numpy as np

    from paper_1911_03813_gb300 import stmf
    opts = dict(pgtol=1e-5, factr=1e9, max_evals=200, alpha_mode=0, chunk=8)
    sat = make_requests(max(n_requests // 4, 8), seed, dev)
    poi = make_requests(n_requests, seed + 1, dev)

    def poisson(srv, rate, draw_seed, reqs=None):
        reqs = poi if reqs is None else reqs
        gaps = np.random.default_rng(draw_seed).exponential(1.0 / rate, size=len(reqs))
        t0 = time.perf_counter()
        due = t0
        tick = []
        for q, gap in zip(reqs, gaps):
            due += gap
            while time.perf_counter() < due:
                time.sleep(0.0002)
            tick.append(srv.submit(q["V"], q["d"], q["x0"], **opts))
        res = [srv.poll(t) for t in tick]
        el = time.perf_counter() - t0
        lat = np.array([r_["t_done"] - r_["t_submit"] for r_ in res]) * 1e3
        return {"arrival_rate_per_s": rate, "fits_per_s": 4 * len(reqs) / el,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "completed": int(sum(r_["state"] == 0 for r_ in res))}

    with stmf.Server(device=device_index, max_fits=64, n_max=128, r_max=16, m_max=5,
                     mem_budget=150 << 30) as srv:
        with UtilSampler(device_index) as u_sat:
            t0 = time.perf_counter()
            tick = [srv.submit(q["V"], q["d"], q["x0"], **opts) for q in sat]
            for t in tick:
                srv.poll(t)
            t_sat = time.perf_counter() - t0
        rate_sat = len(sat) / t_sat
        with UtilSampler(device_index) as u_poi:
            main = poisson(srv, 0.8 * rate_sat, seed + 2)
        main["gpu_busy_pct"] = u_poi.mean()
        extra = []
        for k, mult in enumerate(sweep):
            row = poisson(srv, mult * rate_sat, seed + 3 + k)
            row["rate_over_saturated"] = mult
            extra.append(row)
        fixed = None
        if fixed_rate and fixed_rate < rate_sat:
            fixed = poisson(srv, fixed_rate, seed + 99, poi[:max(len(poi) // 4, 8)])
            fixed["requests"] = max(len(poi) // 4, 8)
        stats = srv.stats()
    out = {"requests": len(poi), "starts_per_request": 4,
           "workload": "n, p log-uniform in [8,128] x [1e3,1e6], d in {3,4}, r in [1,16], "
                       "sigma log-uniform in [1e-4,1e-1], BF16 samples on the host (a pool of "
                       "256 seeded sample sets, request k using set k mod 256)",
           "saturated_requests": len(sat),
           "saturated_requests_per_s": rate_sat, "saturated_fits_per_s": 4 * rate_sat,
           "saturated_gpu_busy_pct": u_sat.mean(),
           "gpu_busy": "nvidia-smi utilization.gpu (share of time some kernel ran), mean of "
                       "100 ms samples over the run",
           **main,
           "peak_admitted_bytes": int(stats["peak_bytes_in_use"]),
           "optimiser": "L-BFGS m=5, pgtol 1e-5, factr 1e9, <= 200 evaluations per start"}
    if extra:
        out["sweep"] = extra
    if fixed is not None:
        out["at_fixed_rate"] = fixed
    return out


def other_passes_bench(st16, st32, lam_t, A_t, dev, only=None, st8=None):
    """The other passes over the samples, on the headline workload's samples (2^24 x 256): the
    range finder of eq. rrf (A0 = V Omega with r_hat = 16, Omega drawn inside the pass; one read
    of the BF16 V, CUDA cores) and the sampled evaluation of Sec. 5 (Lemma 5.1) on 2^20 rows
    gathered at random from the BF16, the FP32 and the E4M3 copy (the tensor-core passes gather
    them), each against the HBM copy peak over the bytes it reads."""
    import torch

    from paper_1911_03813_gb300 import stmf
    peaks = measured_peaks()
    p, n = st16["data"].shape[0], st16["n"]

    def events(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {}
    if only in (None, "rrf"):
        ms_rrf = events(lambda: stmf.rrf_start(st16, 16, 7), 5)
        gb_rrf = p * n * 2 / (ms_rrf / 1e3) / 1e9
        out["rrf_start"] = {"n": n, "p": p, "r_hat": 16, "dtype": "bf16", "ms": ms_rrf,
                            "gbs_over_V": gb_rrf, "frac_of_hbm": gb_rrf / peaks["hbm_gbs"]}
    s = 1 << 20
    idx = torch.randint(0, p, (s,), device=dev, dtype=torch.int64,
                        generator=torch.Generator(device=dev).manual_seed(SEED))
    for name, st, eb in (("sampled_fg_bf16", st16, 2), ("sampled_fg_f32", st32, 4),
                         ("sampled_fg_e4m3", st8, 1)):
        if st is None or only not in (None, name[len("sampled_fg_"):]):
            continue
        ms_smp = events(lambda: stmf.fg_sampled(st, idx, D, lam_t, A_t), 20)
        row_bytes = n * eb + (4 if name.endswith("e4m3") else 0)  # E4M3: codes and the scale
        gb_smp = s * row_bytes / (ms_smp / 1e3) / 1e9
        out[name] = {"n": n, "rows": s, "r": R, "d": D, "ms": ms_smp, "gbs_over_rows": gb_smp,
                     "frac_of_hbm": gb_smp / peaks["hbm_gbs"], "row_draw": "uniform, with replacement"}
    return out


# Sec. 4.1's timing scenarios (Table timing_compare): d, n, p, r and the paper's implicit time per
# inner iteration in seconds (MATLAB on a 28-core CPU; context, not a target)
PAPER_E1 = [(3, 75, 750, 5, 4.36e-4), (3, 75, 750, 25, 5.91e-4), (3, 75, 3750, 5, 7.96e-4),
            (3, 75, 3750, 25, 1.03e-3), (3, 375, 3750, 5, 4.82e-3), (4, 75, 3750, 5, 9.22e-4)]


def paper_shapes_bench(dev, oracle_seconds=1.0):
    """Sec. 4.1's six timing scenarios as a context workload: uniform(0,1) samples in FP64. Per
    scenario: the device's time per f+grad evaluation (200 back to back, CUDA events); a fit on
    the device from a seeded random start with pgtol = 0.05, as in Sec. 4.1 (time per inner
    iteration, the paper's unit); the FP64 oracle's time per evaluation on the host cores; and
    the paper's implicit time per inner iteration beside them."""
    import numpy as np
    import torch

    import oracle
    from paper_1911_03813_gb300 import inputs, stmf
    rows = []
    for k, (d, n, p, r, paper_s) in enumerate(PAPER_E1):
        V = inputs.uniform(n, p, seed=SEED + k)
        st = inputs.to_storage(V, "f64", device=dev)
        lam, A = inputs.random_model(n, r, seed=SEED + 100 + k)
        lam_t = torch.tensor(lam, device=dev)
        A_t = torch.tensor(np.ascontiguousarray(A.T), device=dev).T
        out = (torch.empty(1, dtype=torch.float64, device=dev),
               torch.empty(r, dtype=torch.float64, device=dev),
               torch.empty((r, n), dtype=torch.float64, device=dev).T)
        for _ in range(5):
            stmf.fg(st, None, d, lam_t, A_t, out=out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(200):
            stmf.fg(st, None, d, lam_t, A_t, out=out)
        e1.record()
        torch.cuda.synchronize()
        eval_s = e0.elapsed_time(e1) / 200 / 1e3
        lam_f = lam_t.clone()
        A_f = torch.tensor(np.ascontiguousarray(A.T), device=dev).T  # column-major, updated in place
        t0 = time.perf_counter()
        res = stmf.fit(st, None, d, lam_f, A_f, pgtol=0.05, max_evals=50000)
        fit_s = time.perf_counter() - t0
        Vt = np.ascontiguousarray(V.T)
        t0, ko = time.perf_counter(), 0
        while time.perf_counter() - t0 < oracle_seconds:
            oracle.fg_implicit(None, Vt, lam, A, d)
            ko += 1
        oracle_s = (time.perf_counter() - t0) / ko
        rows.append({"d": d, "n": n, "p": p, "r": r, "gpu_s_per_eval": eval_s,
                     "gpu_fit_s": fit_s, "gpu_fit_evals": res["evals"],
                     "gpu_fit_s_per_iter": fit_s / max(res["evals"], 1),
                     "fit_stop": res["stop_name"], "oracle_s_per_eval": oracle_s,
                     "paper_implicit_s_per_iter": paper_s})
    return {"workload": "Sec. 4.1 scenarios, uniform(0,1) samples, FP64, nu = 1/p",
            "paper_context": "Table timing_compare, implicit method: MATLAB 2018a on 2 x Intel "
                             "E5-2683 (28 cores), L-BFGS-B; per inner iteration",
            "oracle_cores": len(os.sched_getaffinity(0)), "scenarios": rows}


def gram_bench(dev):
    """One ||X||^2 Gram pass (tensor cores, BF16) on the first 2^18 samples of the workload (the
    pass is O(p^2 n): 1.8e13 FLOP here; with 2^16 samples, about 14 work items per CTA, the tail
    and the I-tile reloads show)."""
    import torch

    from paper_1911_03813_gb300 import inputs, stmf
    p = 1 << 18
    st = inputs.gmm_device(N_FEAT, p, N_MEANS, SIGMA, SEED, dev, out_dtype="bf16")
    stmf.norm_x(st, None, D)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    reps = 5
    for _ in range(reps):
        stmf.norm_x(st, None, D)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    T = (p + 127) // 128
    flop = 2.0 * 128 * 128 * N_FEAT * T * (T + 1) / 2
    pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1900.0}
    tf = flop / (ms / 1e3) / 1e12
    return {"p": p, "n": N_FEAT, "d": D, "ms": ms, "tflops": tf, "bound": "tensor",
            "peak_tflops": pk["bf16_tflops"], "frac": tf / pk["bf16_tflops"],
            "flop_counted": "2*128*128*n per computed 128x128 tile pair, upper triangle"}


def alpha_bench(dev):
    """||X||^2 at the FP32 scale workload (n=100, p=2.5e6, 10 means, d=3), two real passes over
    all 2.5e6 samples: the method stmf_norm_x picks for FP32 samples (the distinct entries of the
    symmetric X), and the Gram form nu^T (V^T V)^d nu on the tensor cores over the BF16 copy of
    the same samples (the BF16 values, so its alpha differs from the FP32 one by the rounding)."""
    import torch

    from paper_1911_03813_gb300 import inputs, stmf
    n, p, d = 100, 2500000, 3
    st = inputs.gmm_device(n, p, 10, 0.1, SEED + 7, dev, out_dtype="f32")
    stmf.norm_x(st, None, d)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    a = stmf.norm_x(st, None, d)
    torch.cuda.synchronize()
    t_auto = time.perf_counter() - t0
    ld16 = inputs.padded_ld(n, "bf16")
    data16 = torch.zeros((p, ld16), dtype=torch.bfloat16, device=dev)
    data16[:, :n] = st["data"][:, :n]
    st16 = dict(st, data=data16, dtype="bf16", ld=ld16)
    del st
    torch.cuda.empty_cache()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g = stmf.norm_x(st16, None, d, method="gram")
    e1.record()
    torch.cuda.synchronize()
    ms_gram = e0.elapsed_time(e1)
    T = (p + 127) // 128
    flop = 2.0 * 128 * 128 * n * T * (T + 1) / 2
    del st16
    return {"n": n, "p": p, "d": d,
            "compressed_fp32": {"method": "distinct entries of the symmetric X (FP32 samples)",
                                "s": t_auto, "alpha": a.item()},
            "gram_bf16_tensor_cores": {"method": "Gram form over all sample pairs (BF16 copy)",
                                       "s": ms_gram / 1e3, "alpha": g.item(),
                                       "tflops": flop / (ms_gram / 1e3) / 1e12,
                                       "flop_counted": "2*128*128*n per computed 128x128 tile "
                                                       "pair, upper triangle"}}


def fp32_scale_bench(dev, evals=1000):
    """The FP32 workload at scale: n=100, p=2.5e6 (10 means, sigma=0.1, Dirichlet weights),
    r=10, a timed batch of `evals` evaluations, each at its own random (lambda, A), for d=3 and
    d=4 (CUDA events; the 1 GB of FP32 samples is larger than L2)."""
    import numpy as np
    import torch

    from paper_1911_03813_gb300 import inputs, stmf
    n, p, r = 100, 2500000, 10
    st = inputs.gmm_device(n, p, 10, 0.1, SEED + 11, dev, out_dtype="f32")
    models = [inputs.random_model(n, r, seed=SEED + 100 + k) for k in range(evals)]
    lams = torch.tensor(np.stack([m[0] for m in models]), device=dev)
    As = torch.tensor(np.stack([np.ascontiguousarray(m[1].T) for m in models]), device=dev)
    f = torch.empty(1, dtype=torch.float64, device=dev)
    gl = torch.empty(r, dtype=torch.float64, device=dev)
    GA = torch.empty((r, n), dtype=torch.float64, device=dev).T
    stmf.reserve(st, r)
    out = {}
    for d in (3, 4):
        for k in range(3):
            stmf.fg(st, None, d, lams[k], As[k].T, out=(f, gl, GA))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(evals):
            stmf.fg(st, None, d, lams[k], As[k].T, out=(f, gl, GA))
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / evals
        out["d%d" % d] = {"evals_per_s": 1e3 / ms, "ms_per_eval": ms,
                          "gbs_over_V": p * n * 4 / (ms / 1e3) / 1e9}
    # the FP64 oracle on the host cores at the same workload: a slice of the samples, scaled by p
    # (the evaluation is linear in p)
    import oracle
    ps = 1 << 17
    Vt = np.ascontiguousarray(st["data"][:ps, :n].double().cpu().numpy().T)
    lam0, A0 = models[0]
    t0, k = time.perf_counter(), 0
    while time.perf_counter() - t0 < 4.0:
        oracle.fg_implicit(None, Vt, lam0, A0, 3)
        k += 1
    per_full = (time.perf_counter() - t0) / k * (p / ps)
    out["oracle_d3"] = {"evals_per_s": 1.0 / per_full, "cores": len(os.sched_getaffinity(0)),
                        "sample": "%d of %d samples, %d evaluations in about 4 s, scaled by p"
                                  % (ps, p, k)}
    del st
    return {"n": n, "p": p, "r": r, "dtype": "f32", "evals": evals, **out}


def autograd_bench(dev, calls=50):
    """The differentiation workload: n=64, d=3, r=8, p=1e6 FP32 samples; the autograd.Function
    over (lambda, A) timed per call, forward (the fused pass and the model terms) against
    backward (the stored gradient scaled by the incoming gradient), CUDA events."""
    import torch

    from paper_1911_03813_gb300 import autograd, inputs
    n, p, r, d = 64, 1000000, 8, 3
    st = inputs.gmm_device(n, p, r, 0.1, SEED + 21, dev, out_dtype="f32")
    lam0, A0 = inputs.random_model(n, r, seed=SEED + 22)
    lam = torch.tensor(lam0, device=dev, requires_grad=True)
    A = torch.tensor(A0, device=dev, requires_grad=True)
    for _ in range(3):
        autograd.objective(lam, A, st, None, d).backward()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fwd = bwd = 0.0
    for _ in range(calls):
        lam.grad = None
        A.grad = None
        torch.cuda.synchronize()
        ev[0].record()
        f = autograd.objective(lam, A, st, None, d)
        ev[1].record()
        f.backward()
        ev[2].record()
        torch.cuda.synchronize()
        fwd += ev[0].elapsed_time(ev[1])
        bwd += ev[1].elapsed_time(ev[2])
    del st
    return {"n": n, "p": p, "r": r, "d": d, "dtype": "f32", "calls": calls,
            "forward_ms": fwd / calls, "backward_ms": bwd / calls,
            "backward_over_forward": bwd / fwd}


METRIC = "f+grad evaluations/s (BF16 V; FP32 V beside it)"


def workload_config(P, world):
    return {"workload": WORKLOAD if P == P_FULL else "gmm_n256_d4_r16_p%d" % P,
            "n": N_FEAT, "d": D, "r": R, "p": P, "sigma": SIGMA,
            "l2": "inputs larger than L2 (8.6 GB BF16 per step)",
            "parallelism": "replicas" if world > 1 else "single"}


def run_reference(args):
    """The FP64 oracle on the host cores. Each step is one evaluation of Alg. 2 on a bounded
    sample of the workload (the first 2^16 of its 2^24 samples, the same seeded mixture):
    ms_per_step is the measured time of that step, and value converts it to evaluations of the
    whole workload per second by the ratio of samples (the evaluation is linear in p)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    import numpy as np

    import oracle
    from paper_1911_03813_gb300 import inputs
    p_sample = 1 << 16
    data = inputs.gmm(N_FEAT, p_sample, N_MEANS, SIGMA, seed=SEED)
    Vt = np.ascontiguousarray(data["V"].T)
    lam, A = inputs.random_model(N_FEAT, R, seed=SEED + 1)
    for _ in range(warm):
        oracle.fg_implicit(None, Vt, lam, A, D)
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.fg_implicit(None, Vt, lam, A, D)
    el = time.perf_counter() - t0
    step_s = el / steps
    v = (p_sample / P_FULL) / step_s
    cfg = workload_config(P_FULL, 1)
    cfg["timed_sample_p"] = p_sample
    sample = ("each step: the FP64 oracle (NumPy) on the first %d of the %d samples; value = "
              "evaluations of the whole workload per second = (%d / %d) / step time"
              % (p_sample, P_FULL, p_sample, P_FULL))
    line = {"impl": "reference", "metric": METRIC, "value": v,
            "unit": "evals/s", "n_gpus": args.gpus, "steps": steps, "warmup": warm,
            "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": v, "unit": "evals/s", "cores": len(os.sched_getaffinity(0)),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def sweep_of(args):
    return tuple(float(x) for x in args.serving_sweep.split(",") if x.strip())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--p", type=int, default=P_FULL)
    ap.add_argument("--serving-requests", type=int, default=4096)
    ap.add_argument("--no-gram", action="store_true")
    ap.add_argument("--serving-sweep", default="",
                    help="comma-separated multiples of the saturated serving rate to run after "
                         "the 0.8x run (e.g. 0.5,1.0,1.2)")
    ap.add_argument("--serving-only", action="store_true",
                    help="only the serving workload (its JSON object on one line)")
    ap.add_argument("--gmm-study", action="store_true",
                    help="run the Gaussian-mixture study grid of Sec. 4.2 (n=500) and print its line")
    ap.add_argument("--alpha-only", action="store_true",
                    help="only ||X||^2 from the distinct entries of X at n=100, p=2.5e6, d=3")
    ap.add_argument("--other-passes-only", choices=["all", "rrf", "bf16", "f32", "e4m3"],
                    default=None,
                    help="time only the range finder and/or the sampled evaluation on --p samples")
    ap.add_argument("--paper-shapes-only", action="store_true",
                    help="time only Sec. 4.1's six scenarios (FP64) and print them")
    ap.add_argument("--gram-only", action="store_true",
                    help="time only the ||X||^2 Gram pass on 2^18 samples and print it")
    ap.add_argument("--legs", default="bf16,fp32,fp8",
                    help="sample types to time (bf16 is the headline)")
    ap.add_argument("--oracle-one-core", nargs=2, type=float, default=None,
                    help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_one_core:
        return oracle_one_core_main(int(args.oracle_one_core[0]), args.oracle_one_core[1])
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1911_03813_gb300 import inputs, stmf

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.paper_shapes_only:
        print(json.dumps(paper_shapes_bench(dev)), flush=True)
        return
    if args.other_passes_only:
        import numpy as np
        import torch

        from paper_1911_03813_gb300 import inputs
        which = None if args.other_passes_only == "all" else args.other_passes_only
        st16 = (inputs.gmm_device(N_FEAT, args.p, N_MEANS, SIGMA, SEED, dev, out_dtype="bf16")
                if which in (None, "rrf", "bf16") else None)
        st32 = (inputs.gmm_device(N_FEAT, args.p, N_MEANS, SIGMA, SEED, dev, out_dtype="f32")
                if which in (None, "f32") else None)
        st8 = (inputs.gmm_device(N_FEAT, args.p, N_MEANS, SIGMA, SEED, dev, out_dtype="e4m3")
               if which in (None, "e4m3") else None)
        lam, A = inputs.random_model(N_FEAT, R, seed=SEED + 1)
        lam_t = torch.tensor(lam, device=dev)
        A_t = torch.tensor(np.ascontiguousarray(A.T), device=dev).T
        first = next(x for x in (st16, st32, st8) if x is not None)  # its p and n
        print(json.dumps(other_passes_bench(st16 if st16 is not None else first, st32, lam_t,
                                            A_t, dev, only=which, st8=st8)), flush=True)
        return
    if args.gram_only:
        print(json.dumps(gram_bench(dev)), flush=True)
        return
    if args.alpha_only:
        print(json.dumps(alpha_bench(dev)), flush=True)
        return
    if args.serving_only:
        print(json.dumps(serving_bench(max(args.serving_requests, 8), SEED, dev, local,
                                       sweep_of(args))), flush=True)
        return
    if args.gmm_study:
        from paper_1911_03813_gb300 import study
        rows, wall = study.run()
        keep = ("d", "r", "sigma", "r_hat", "rel_error", "score", "evals", "stop")
        fits = len(rows) * 10
        print(json.dumps({"metric": "Gaussian-mixture study of Sec. 4.2 (n=500, p=250r, "
                                    "r_hat in r-2..r+2, best of 10 RRF starts, pgtol 1e-4)",
                          "value": fits / wall, "unit": "fits/s", "fits": fits, "wall_s": wall,
                          "dtype": "f32", "data": "synthetic",
                          "rows": [{k: row[k] for k in keep} for row in rows]}), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    P = args.p
    legs = args.legs.split(",")
    if "fp32" in legs:
        st32 = inputs.gmm_device(N_FEAT, P, N_MEANS, SIGMA, SEED + rank, dev, out_dtype="f32")
        st16 = dict(st32)
        st16["data"] = st32["data"].to(torch.bfloat16)
        st16["dtype"] = "bf16"
        st16["ld"] = inputs.padded_ld(N_FEAT, "bf16")
    else:
        st16 = inputs.gmm_device(N_FEAT, P, N_MEANS, SIGMA, SEED + rank, dev, out_dtype="bf16")
        st32 = None
    st8 = None
    if "fp8" in legs:
        st8 = inputs.gmm_device(N_FEAT, P, N_MEANS, SIGMA, SEED + rank, dev, out_dtype="e4m3")
    lam, A = inputs.random_model(N_FEAT, R, seed=SEED + 1)
    lam_t = torch.tensor(lam, device=dev)
    A_t = torch.tensor(A.T.copy(), device=dev).T
    ctx = stmf.default_context(local)
    stmf.reserve(st16, R)
    if st32 is not None:
        stmf.reserve(st32, R)
    if st8 is not None:
        stmf.reserve(st8, R)
    f = torch.empty(1, dtype=torch.float64, device=dev)
    gl = torch.empty(R, dtype=torch.float64, device=dev)
    GA = torch.empty((R, N_FEAT), dtype=torch.float64, device=dev).T
    out = (f, gl, GA)
    stream = torch.cuda.current_stream()

    def timed(st, steps, warm, prof=False):
        for _ in range(warm):
            stmf.fg(st, None, D, lam_t, A_t, out=out)
        if prof:
            stmf.profile_enable(True, ctx=ctx)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            stmf.fg(st, None, D, lam_t, A_t, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        pass_ms = None
        if prof:
            tot, cnt = stmf.profile_read(ctx=ctx)
            stmf.profile_enable(False, ctx=ctx)
            pass_ms = tot / max(cnt, 1)
        return ms, pass_ms

    if "fp32" in legs:
        ms32, pass32 = timed(st32, max(args.steps // 2, 1), args.warmup, prof=True)
    else:
        ms32 = pass32 = float("nan")
    ms8 = pass8 = float("nan")
    if st8 is not None:
        ms8, pass8 = timed(st8, args.steps, args.warmup, prof=True)
    with ClockSampler(local) as clk:
        ms16, pass16 = timed(st16, args.steps, args.warmup, prof=True)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms16, ms32], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms16, ms32 = t.tolist()
    steps32 = max(args.steps // 2, 1)
    value = world * args.steps / (ms16 / 1e3)
    bytes16 = P * N_FEAT * 2
    bytes32 = P * N_FEAT * 4
    peaks = measured_peaks()
    ach16 = bytes16 / (pass16 / 1e3) / 1e9
    ach32 = bytes32 / (pass32 / 1e3) / 1e9

    # end to end through the public API with host buffers: stmf_fg_host streams V from pinned
    # host memory in chunks (copies overlapped with the passes) and returns f and g to the host
    e2e = None
    if args.e2e_steps > 0:
        host16 = torch.empty(st16["data"].shape, dtype=torch.bfloat16, pin_memory=True)
        host16.copy_(st16["data"])
        st_h = dict(st16)
        st_h["data"] = host16
        lam_h = lam.copy()
        A_h = np.asfortranarray(A)
        for _ in range(3):
            stmf.fg_host(st_h, None, D, lam_h, A_h)
        barrier()
        calls = []
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            tc = time.perf_counter()
            stmf.fg_host(st_h, None, D, lam_h, A_h)
            calls.append(time.perf_counter() - tc)
        el = time.perf_counter() - t0
        barrier()
        # the host-to-device link's own copy rate (one pinned 1 GiB copy, CUDA events): the
        # end-to-end call moves V over this link every step, so it bounds the e2e rate
        lk_h = torch.empty(1 << 30, dtype=torch.uint8, pin_memory=True)
        lk_d = torch.empty(1 << 30, dtype=torch.uint8, device=dev)
        lk_d.copy_(lk_h, non_blocking=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            lk_d.copy_(lk_h, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        link_gbs = 3 * (1 << 30) / (e0.elapsed_time(e1) * 1e-3) / 1e9
        del lk_h, lk_d
        h2d_gbs = (bytes16 + 8 * (R + R * N_FEAT + 1)) * args.e2e_steps / el / 1e9
        e2e = {"value": world * args.e2e_steps / el, "unit": "evals/s",
               "h2d_gbs": round(h2d_gbs, 1), "link_h2d_gbs_measured": round(link_gbs, 1),
               "link_frac": round(h2d_gbs / link_gbs, 3),
               "h2d_bytes_per_step": bytes16 + 8 * (R + R * N_FEAT + 1),
               "d2h_bytes_per_step": 8 * (1 + R + R * N_FEAT),
               "calls_ms": [round(1e3 * c, 2) for c in calls],
               "call_ms_median": round(1e3 * statistics.median(calls), 2),
               "call_ms_min": round(1e3 * min(calls), 2),
               "call": "stmf_fg_host (pinned host V, chunked H2D overlapped with the passes)"}
        del host16, st_h

    if rank != 0:
        return
    other = None if args.no_gram else other_passes_bench(st16, st32, lam_t, A_t, dev, st8=st8)
    del st16, st32, st8
    torch.cuda.empty_cache()
    gram = None if args.no_gram else gram_bench(dev)
    alpha = None if args.no_gram else alpha_bench(dev)
    fp32_scale = None if args.no_gram else fp32_scale_bench(dev)
    differentiation = None if args.no_gram else autograd_bench(dev)
    paper_shapes = None if args.no_gram else paper_shapes_bench(dev)
    serving = (serving_bench(args.serving_requests, SEED, dev, local, sweep_of(args))
               if args.serving_requests else None)
    cpu = None if args.no_cpu_baseline else cpu_baseline(dev)
    traffic = ncu_traffic("fg_pass_bf16")
    line = {
        "metric": METRIC,
        "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms16 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": workload_config(P, world),
        "hbm_gbs_over_V": bytes16 / (ms16 / args.steps / 1e3) / 1e9,
        "roofline": {"bound": "hbm", "achieved": ach16, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": ach16 / peaks["hbm_gbs"], "traffic": traffic,
                     "kernel": "fused pass (Alg. 2: Y and w)", "peak_src": peaks["src"],
                     "algorithmic_bytes_per_launch": bytes16},
        "fp32": {"value": steps32 / (ms32 / 1e3) * world, "unit": "evals/s",
                 "ms_per_step": ms32 / steps32, "hbm_gbs_over_V": bytes32 / (ms32 / steps32 / 1e3) / 1e9,
                 "pass_frac_of_hbm": ach32 / peaks["hbm_gbs"],
                 "roofline": {"bound": "hbm", "achieved": ach32, "peak": peaks["hbm_gbs"],
                              "unit": "GB/s", "frac": ach32 / peaks["hbm_gbs"],
                              "traffic": ncu_traffic("fg_pass_f32"),
                              "kernel": "fused pass, FP32 samples (tensor cores, in-place "
                                        "BF16 hi/lo split)",
                              "peak_src": peaks["src"],
                              "algorithmic_bytes_per_launch": bytes32},
                 "bf16_over_fp32": (args.steps / ms16) / (steps32 / ms32)},
        "fp8": {"value": args.steps / (ms8 / 1e3) * world, "unit": "evals/s",
                "ms_per_step": ms8 / args.steps,
                "pass_gbs_over_V": P * (N_FEAT + 4) / (pass8 / 1e3) / 1e9,
                "pass_frac_of_hbm": P * (N_FEAT + 4) / (pass8 / 1e3) / 1e9 / peaks["hbm_gbs"],
                "storage": "E4M3 codes + one FP32 scale per sample"},
        "clocks": clk.summary(),
        "gpu_launches": 3 * args.steps,
        "e2e": e2e,
        "gram": gram,
        "paper_shapes": paper_shapes,
        "other_passes": other,
        "alpha_fp32_scale": alpha,
        "fp32_scale": fp32_scale,
        "differentiation": differentiation,
        "serving": serving,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
