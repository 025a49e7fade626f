#!/usr/bin/env python
"""Benchmark: batched negacyclic NTT KOPS at N = 2^16 and CKKS HMULT KOPS on one GB300.

Workload of `value` (one step): forward NTT + inverse NTT, in place, of 64 polynomials x 44
RNS limbs (30-bit primes q_0..q_43) at N = 2^16 -- one fhe_ntt_fwd and one fhe_ntt_inv call
(704 MiB resident in HBM, larger than L2, so no flush is needed between steps). One op = one
limb transform (the #NTT/s unit of Table VIII). The JSON line also carries both NTT paths,
the HMULT throughput (N = 2^16, 24 + 8 limbs, dnum = 3, 128 ciphertext pairs per call), the
end-to-end number through the C ABI with host buffers, the roofline of the dominant kernel
and the CPU oracle timed on this host.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs the same per-GPU workload on its own GPU (replicas;
the path has no exchange step) and rank 0 prints the aggregate.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2212_14191_gb300 import configs as CFG  # noqa: E402  (after the path insert)

METRIC = "NTT KOPS and HMULT KOPS at N=2^16 (INT8-TC vs plain CUDA), % INT8/HBM roofline"
LOGN, N = CFG.NTT_FULL.logN, 1 << CFG.NTT_FULL.logN
NTT_LIMBS, NTT_BATCH = CFG.NTT_FULL.limbs, CFG.NTT_FULL.batch
HM_LIMBS, HM_K, HM_ALPHA, HM_BATCH = (CFG.HMULT_FULL.limbs, CFG.HMULT_FULL.special, CFG.HMULT_FULL.alpha,
                                      CFG.HMULT_FULL.batch)
E2E_LIMBS = 11  # limbs per chunk of the pipelined end-to-end step


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--hmult-steps", type=int, default=3)
    ap.add_argument("--no-hmult", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default plain-path variants (for profiling runs)")
    ap.add_argument("--paths", default="u32,tc", help="NTT paths to time: u32, tc or both")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-heax", action="store_true", help="skip the HEAX comparison parameter sets")
    ap.add_argument("--serving-seconds", type=float, default=2.0, help="seconds of arrivals per serving run")
    ap.add_argument("--batch-ops", type=int, default=1000)
    ap.add_argument("--e2e-limbs", type=int, default=E2E_LIMBS, help="limbs per chunk of the end-to-end pipeline")
    ap.add_argument("--ntt-batch", type=int, default=NTT_BATCH,
                    help="polynomials per limb of the NTT step (smaller for counter captures)")
    ap.add_argument("--hmult-batch", type=int, default=HM_BATCH,
                    help="ciphertext pairs per HMULT call (and ciphertexts per HROTATE / CMULT / HADD call)")
    return ap.parse_args()


def dist_env():
    from paper_2212_14191_gb300 import replicas
    return replicas.dist_env()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi every 50 ms while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def variant_name(v):
    """NTT variant (see ntt_u32.cu; 32 and 33 are the tensor-core path) in words."""
    if v >= 32:
        return "variant %d: tensor-core path, %d-column output tiles" % (v, 64 if v == 32 else 32)
    shape = "512-thread CTAs" if v & 1 == 0 else "256-thread CTAs"
    ex = ["pull clusters", "push clusters", "split-forward clusters",
          "two-pass via L2 (decimation-in-time forward)"][(v >> 1) & 3]
    extra = (", staged twiddles" if v & 8 else "") + (", 64 registers" if v & 16 else "")
    return "variant %d: %s, %s%s" % (v, shape, ex, extra)


def traffic_for(kernel_file, key):
    """Per-launch DRAM bytes of a kernel from a committed ncu summary, if still current."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(key)
        with open(os.path.join(ROOT, kernel_file), "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()[:16]
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_sha256_16") != h:
        return None
    return rec.get("dram_bytes_per_launch")


# ------------------------------------------------------------------ CPU oracle (baseline leg)


def cpu_oracle_kops(budget_s=10.0, batch_cap=NTT_BATCH):
    """The C oracle (oracle/ntt_oracle.c, OpenMP over rows, as it stands) on a bounded
    sample of the same workload: all 44 limbs x b polynomials, forward + inverse."""
    from oracle import ntt as ON
    from oracle import params as P
    from paper_2212_14191_gb300 import inputs as I
    qs, _ = P.default_moduli(NTT_LIMBS, 8)
    psis = [P.psi(q, N) for q in qs]
    b = 1
    while True:
        x = I.uniform_residues(5, qs, b, N)
        t0 = time.perf_counter()
        y, used = ON.ntt_batch(x, qs, psis)
        z, _ = ON.ntt_batch(y, qs, psis, inverse=True)
        dt = time.perf_counter() - t0
        assert (z == x).all()
        if dt * 2 > budget_s or b * 2 > batch_cap:
            ops = 2 * NTT_LIMBS * b
            # the same oracle on one thread, on one polynomial per limb
            x1 = x[:, :1, :]
            t1 = time.perf_counter()
            y1, _ = ON.ntt_batch(x1, qs, psis, threads=1)
            ON.ntt_batch(y1, qs, psis, inverse=True, threads=1)
            dt1 = time.perf_counter() - t1
            return {"value": ops / dt / 1e3, "unit": "KOPS", "cores": used, "kind": "oracle",
                    "sample": "%d limbs x %d polys, fwd+inv NTT at N=2^16 (%d limb transforms, %.1f s)"
                              % (NTT_LIMBS, b, ops, dt),
                    "single_thread": {"value": 2 * NTT_LIMBS / dt1 / 1e3, "unit": "KOPS", "cores": 1,
                                      "sample": "%d limbs x 1 poly, fwd+inv (%.2f s)" % (NTT_LIMBS, dt1)},
                    "host": host_cpu()}
        b *= 2


def cpu_oracle_hmult(budget_s=8.0, n=N):
    """The CKKS oracle (oracle/ckks.py: numpy, with the C oracle's transforms, as it stands) on
    one ciphertext pair of the HMULT workload (24 + 8 limbs, dnum = 3): HMULT with
    relinearisation and rescale, repeated until half the budget is spent. Context only: the
    oracle exists to check parity. Random residues stand in for the key (timing does not
    depend on the values)."""
    from oracle import ckks as C
    from oracle import params as P
    from paper_2212_14191_gb300 import inputs as I
    qs, ps = P.default_moduli(HM_LIMBS, HM_K)
    prm = C.Params(n, qs, ps, alpha=HM_ALPHA)
    dnum = prm.dnum(HM_LIMBS)
    ct = [I.uniform_residues(20 + i, qs, 2, n, dtype=np.uint64).transpose(1, 0, 2) for i in range(2)]
    evk = I.uniform_residues(22, qs + ps, dnum * 2, n, dtype=np.uint64).reshape(
        HM_LIMBS + HM_K, dnum, 2, n).transpose(1, 2, 0, 3)
    done, t0 = 0, time.perf_counter()
    while True:
        out = C.hmult(prm, HM_LIMBS, ct[0], ct[1], evk)
        done += 1
        dt = time.perf_counter() - t0
        if dt * 2 > budget_s:
            break
    assert out.shape == (2, HM_LIMBS - 1, n)
    return {"value": done / dt / 1e3, "unit": "KOPS (HMULT + relinearisation + rescale)", "kind": "oracle",
            "cores": "numpy on one thread, transforms on up to %d" % (os.cpu_count() or 1),
            "sample": "%d ciphertext pair(s), N=%d, %d + %d limbs, dnum=%d (%.1f s)"
                      % (done, n, HM_LIMBS, HM_K, dnum, dt)}


def host_cpu():
    """CPU model and logical core count of this host, from /proc/cpuinfo where it says."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
        for key in ("model name", "Model", "CPU part"):
            for line in info.splitlines():
                if line.split(":")[0].strip() == key:
                    model = line.split(":", 1)[1].strip()
                    break
            if model:
                model = ("CPU part " + model) if key == "CPU part" else model
                break
    except OSError:
        pass
    import platform
    return "%s, %s, %d logical cores" % (model or "unknown model", platform.machine(), os.cpu_count() or 0)


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import ntt as ON
    from oracle import params as P
    from paper_2212_14191_gb300 import inputs as I
    qs, _ = P.default_moduli(NTT_LIMBS, 8)
    psis = [P.psi(q, N) for q in qs]
    b = 2  # each step: 44 limbs x 2 polynomials, forward + inverse (a bounded sample)
    x = I.uniform_residues(5, qs, b, N)
    used = 1
    for _ in range(args.warmup):
        y, used = ON.ntt_batch(x, qs, psis)
        ON.ntt_batch(y, qs, psis, inverse=True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        y, used = ON.ntt_batch(x, qs, psis)
        ON.ntt_batch(y, qs, psis, inverse=True)
    dt = time.perf_counter() - t0
    ops = 2 * NTT_LIMBS * b * args.steps
    v = ops / dt / 1e3
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "KOPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": "batched NTT+INTT, N=2^16, 44 limbs, per step 2 polynomials (sample of 64)",
                   "timing": "host wall clock"},
        "cpu_baseline": {"value": v, "unit": "KOPS", "cores": used, "kind": "oracle",
                         "sample": "44 limbs x 2 polys fwd+inv per step at N=2^16"},
        "e2e": {"value": v, "unit": "KOPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------ GPU arm


def ours(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2212_14191_gb300 import fhe
    from paper_2212_14191_gb300 import inputs as I
    from paper_2212_14191_gb300 import replicas as R
    R.init(ws, "nccl", torch.device("cuda", local))

    def barrier():
        R.barrier(ws)

    def max_over_ranks(v):
        return R.max_over_ranks(v, ws)

    allp = fhe.fhe_gen_primes(16, 30, NTT_LIMBS + 8)
    ps, qs = allp[:8], allp[8:]
    ctx = fhe.Context(16, qs, ps, alpha=HM_ALPHA, default_path=fhe.FHE_NTT_U32)
    st = torch.cuda.current_stream()
    sh = st.cuda_stream
    x_host = I.uniform_residues(R.rank_seed(1234, rank), qs, NTT_BATCH, N)
    x = fhe.to_device(x_host)
    ops_per_step = 2 * NTT_LIMBS * NTT_BATCH

    def step(path, ev=None):
        if ev is not None:
            ev[0].record(st)
        fhe.fhe_ntt_fwd(ctx.handle, path, LOGN, x.data_ptr(), 0, NTT_LIMBS, NTT_BATCH, sh)
        if ev is not None:
            ev[1].record(st)
        fhe.fhe_ntt_inv(ctx.handle, path, LOGN, x.data_ptr(), 0, NTT_LIMBS, NTT_BATCH, sh)
        if ev is not None:
            ev[2].record(st)

    def time_path(path, steps, warmup):
        for _ in range(warmup):
            step(path)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        # NVTX ranges name the timed regions for profilers (ncu --nvtx --nvtx-include "ntt_u32/")
        torch.cuda.nvtx.range_push("ntt_u32" if path == fhe.FHE_NTT_U32 else "ntt_tc")
        t0.record(st)
        for i in range(steps):
            step(path, evs[i])
        t1.record(st)
        torch.cuda.nvtx.range_pop()
        barrier()
        total = t0.elapsed_time(t1) / 1e3
        fwd = statistics.mean(e[0].elapsed_time(e[1]) for e in evs) / 1e3
        inv = statistics.mean(e[1].elapsed_time(e[2]) for e in evs) / 1e3
        return max_over_ranks(total), fwd, inv

    # the library's autotuner picks the plain-path variant of each direction for this workload
    tune_fwd = tune_inv = None
    if not args.no_autotune:
        tune_fwd, tune_inv = fhe.fhe_autotune_ntt(ctx.handle, LOGN, x.data_ptr(), NTT_LIMBS, NTT_BATCH, reps=2,
                                                  stream=sh)
    x.copy_(fhe.to_device(x_host))
    paths = {k: v for k, v in (("u32", fhe.FHE_NTT_U32), ("tc", fhe.FHE_NTT_TC)) if k in args.paths.split(",")}
    results = {}
    clocks = None
    for name, path in paths.items():
        with ClockSampler(local) as cs:
            total, fwd, inv = time_path(path, args.steps, args.warmup)
        if clocks is None or name == "u32":
            clocks = cs.summary()
        results[name] = {"kops": R.whole_job_rate(ops_per_step * args.steps, ws, total) / 1e3,
                         "fwd_ms": fwd * 1e3, "inv_ms": inv * 1e3}
    vf, vi = fhe.fhe_ntt_get_variant(ctx.handle, LOGN, 0), fhe.fhe_ntt_get_variant(ctx.handle, LOGN, 1)
    if "u32" in results:
        results["u32"]["autotune_ms"] = None if tune_fwd is None else {
            "fwd": [round(v, 4) for v in tune_fwd], "inv": [round(v, 4) for v in tune_inv]}
        results["u32"]["variant"] = {"fwd": vf, "inv": vi}
    fhe.fhe_device_status(ctx.handle, 1)
    head = max(results, key=lambda k: results[k]["kops"])
    # kernels per step: u32 = one launch per direction (per 1 GiB chunk of rows for the
    # two-pass variants); tensor cores = 3 per chunk of limbs and direction (split, GEMM 1,
    # GEMM 2)
    chunk_limbs = max(1, min(64, (256 << 20) // (N * 8) // NTT_BATCH))

    def u32_launches(v):
        rows = NTT_LIMBS * NTT_BATCH
        return (-(-rows // ((1 << 30) // (N * 4 + 4)))) if ((v >> 1) & 3) == 3 else 1   # 1 GiB chunks

    launches_per_step = {"u32": u32_launches(vf) + u32_launches(vi), "tc": 2 * 3 * (-(-NTT_LIMBS // chunk_limbs))}
    total_head = ops_per_step * args.steps * ws / (results[head]["kops"] * 1e3)
    # end to end through the C ABI with host buffers: every step copies the 44 x 64 batch in
    # from pinned host memory, transforms it forward and back, and copies it out. The batch
    # moves in chunks of --e2e-limbs limbs on three streams (H2D, compute, D2H) so that the two
    # copy directions and the kernels overlap; every step still moves all of its bytes.
    pinned_in = torch.from_numpy(x_host.view(np.int32)).pin_memory()
    pinned_out = torch.empty_like(pinned_in).pin_memory()
    e2e_steps = max(2, args.steps // 2)
    s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    el = max(1, args.e2e_limbs)
    chunks = [(l0, min(NTT_LIMBS, l0 + el)) for l0 in range(0, NTT_LIMBS, el)]
    # two device buffers, alternate steps: a chunk's copy-in waits for the copy-out of the
    # same chunk two steps back, not the previous step's
    xbufs = [x, torch.empty_like(x)]
    ev_in = [torch.cuda.Event() for _ in chunks]
    ev_cmp = [torch.cuda.Event() for _ in chunks]
    ev_out = [[torch.cuda.Event() for _ in chunks] for _ in xbufs]
    barrier()
    for evs in ev_out:
        for e in evs:
            e.record(s_out)
    e2e_count = [0]

    def e2e_step(path):
        b = e2e_count[0] & 1
        e2e_count[0] += 1
        xb = xbufs[b]
        for c, (l0, l1) in enumerate(chunks):
            s_in.wait_event(ev_out[b][c])       # this buffer's copy-out of the chunk is done
            with torch.cuda.stream(s_in):
                xb[l0:l1].copy_(pinned_in[l0:l1], non_blocking=True)
            ev_in[c].record(s_in)
            s_cmp.wait_event(ev_in[c])
            fhe.fhe_ntt_fwd(ctx.handle, path, LOGN, xb[l0:l1].data_ptr(), l0, l1 - l0, NTT_BATCH, s_cmp.cuda_stream)
            fhe.fhe_ntt_inv(ctx.handle, path, LOGN, xb[l0:l1].data_ptr(), l0, l1 - l0, NTT_BATCH, s_cmp.cuda_stream)
            ev_cmp[c].record(s_cmp)
            s_out.wait_event(ev_cmp[c])
            with torch.cuda.stream(s_out):
                pinned_out[l0:l1].copy_(xb[l0:l1], non_blocking=True)
            ev_out[b][c].record(s_out)

    for _ in range(2):
        e2e_step(paths[head])
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("e2e")
    e0.record(s_in)
    for _ in range(e2e_steps):
        e2e_step(paths[head])
    e1.record(s_out)                            # after the last copy-out, which follows all work
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    e2e_t = max_over_ranks(e0.elapsed_time(e1) / 1e3)
    assert np.array_equal(pinned_out.numpy().view(np.uint32), x_host)
    nbytes = x_host.nbytes

    # HMULT (N = 2^16, 24 + 8 limbs, dnum = 3, 128 pairs): uniform ciphertexts and key
    hm = ops = None
    if not args.no_hmult:
        hb = args.hmult_batch
        a = fhe.to_device(I.uniform_residues(11, qs[:HM_LIMBS], 2 * hb, N))
        b = fhe.to_device(I.uniform_residues(12, qs[:HM_LIMBS], 2 * hb, N))
        a = a.view(HM_LIMBS, 2, hb, N).permute(1, 0, 2, 3).contiguous()
        b = b.view(HM_LIMBS, 2, hb, N).permute(1, 0, 2, 3).contiguous()
        dnum = -(-HM_LIMBS // HM_ALPHA)
        evk = fhe.to_device(I.uniform_residues(13, qs[:HM_LIMBS] + ps, 2 * dnum, N)).view(
            HM_LIMBS + HM_K, dnum, 2, N).permute(1, 2, 0, 3).contiguous()
        out = torch.empty((2, HM_LIMBS - 1, hb, N), dtype=torch.int32, device="cuda")
        hm = {"config": "N=2^16, 24 ciphertext limbs + 8 special primes, dnum=3, %d pairs per call, " % hb +
                        "HMULT + relinearisation + rescale"}
        for name, path in (("u32", fhe.FHE_NTT_U32), ("tc", fhe.FHE_NTT_TC)):
            hctx = fhe.Context(16, qs[:HM_LIMBS], ps, alpha=HM_ALPHA, default_path=path)
            if path == fhe.FHE_NTT_U32:
                fhe.fhe_ntt_set_variant(hctx.handle, LOGN, fhe.fhe_ntt_get_variant(ctx.handle, LOGN, 0),
                                        fhe.fhe_ntt_get_variant(ctx.handle, LOGN, 1))
            hctx.hmult(a, b, evk, LOGN, out=out)
            barrier()
            h0 = torch.cuda.Event(enable_timing=True)
            h1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.nvtx.range_push("hmult_" + name)
            h0.record(st)
            for _ in range(args.hmult_steps):
                hctx.hmult(a, b, evk, LOGN, out=out)
            h1.record(st)
            torch.cuda.nvtx.range_pop()
            barrier()
            fhe.fhe_device_status(hctx.handle, 1)
            ht = max_over_ranks(h0.elapsed_time(h1) / 1e3)
            # fully fused HBM floor per op: both input ciphertexts, the output, evk / batch
            dnum_h = -(-HM_LIMBS // HM_ALPHA)
            op_bytes = (16 * HM_LIMBS + 8 * (HM_LIMBS - 1)) * N + dnum_h * 2 * (HM_LIMBS + HM_K) * N * 4 / hb
            kops = hb * args.hmult_steps * ws / ht / 1e3
            ceil_kops = measured_peaks()[0]["hbm_gbs"] * 1e9 / op_bytes / 1e3
            hm[name] = {"kops": kops, "ms_per_call": ht / args.hmult_steps * 1e3,
                        "hbm_floor_bytes_per_op": op_bytes, "hbm_ceiling_kops": ceil_kops,
                        "frac_of_hbm_ceiling": kops / ceil_kops}
            if path == fhe.FHE_NTT_U32:
                ops = other_ops(args, fhe, hctx, a, b, evk, st, barrier, max_over_ranks, ws)
            hctx.close()
            del hctx
            torch.cuda.empty_cache()
        del a, b, evk, out

    batch_res = None if args.no_batch else mixed_batch(args, fhe, ctx, qs, ps, st, barrier, max_over_ranks, ws)

    serve_res = None if args.no_serving else serving_bench(args, fhe, qs, ps)

    heax_res = None if args.no_heax else heax_sets(args, fhe, st, barrier, max_over_ranks, ws)

    if rank == 0:
        peaks, peak_kind = measured_peaks()
        n1, n2 = 1 << ((LOGN + 1) // 2), 1 << (LOGN // 2)
        rows = NTT_LIMBS * NTT_BATCH
        roof_u32 = roof_alu = roof_imad = roof_tc = None
        if "u32" in results:
            u32_bytes = 8 * N * rows   # read + write N u32 per limb transform
            u32_gbs = u32_bytes / (results["u32"]["fwd_ms"] / 1e3) / 1e9
            roof_u32 = {"bound": "hbm", "achieved": u32_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": u32_gbs / peaks["hbm_gbs"], "peak_kind": peak_kind,
                        "kernel": "forward plain NTT call at N=2^16 (%s), %d launch(es) per call"
                                  % (variant_name(vf), u32_launches(vf)),
                        "traffic": traffic_for("paper_2212_14191_gb300/csrc/" +
                                               ("ntt_u32_l2.cuh" if ((vf >> 1) & 3) == 3 else "ntt_u32_kernels.cuh"),
                                               "ntt_fwd_u32_n65536_v%d" % vf)}
            # the plain NTT is bound by integer instruction issue, not HBM. A Harvey butterfly is
            # at least 6 integer instructions on sm_103a (the Shoup product: mul.hi and two
            # mul.lo; the conditional subtraction of 2q as one add-min; the two outputs: add,
            # subtract-add), (N/2) log2 N butterflies per limb transform. Peak: 152 SMs x 4
            # schedulers x one 32-lane warp instruction per clock x the maximum SM clock.
            sm_mhz = (clocks or {}).get("sm_max_mhz") or 2070
            fwd_s = results["u32"]["fwd_ms"] / 1e3
            issue_peak = 152 * 4 * 32 * sm_mhz * 1e6 / 1e12
            alu_ach = 6 * (N // 2) * LOGN * rows / fwd_s / 1e12
            roof_alu = {"bound": "alu", "achieved": alu_ach, "peak": issue_peak, "unit": "T int-instr/s",
                        "frac": alu_ach / issue_peak,
                        "peak_kind": "derived: 152 SMs x 4 schedulers x 32 lanes x max SM clock",
                        "kernel": roof_u32["kernel"], "traffic": roof_u32["traffic"],
                        "note": "algorithmic work = 6 integer instructions per radix-2 butterfly "
                                "(3 for the Shoup product, 3 add/min) x (N/2) log2 N butterflies per limb transform"}
            # the multiply pipe alone: 3 IMAD per Shoup product, 64 IMAD lanes per clock per SM
            imad_peak = 152 * 64 * sm_mhz * 1e6 / 1e12
            imad_ach = 3 * (N // 2) * LOGN * rows / fwd_s / 1e12
            roof_imad = {"bound": "alu", "achieved": imad_ach, "peak": imad_peak, "unit": "T IMAD/s",
                         "frac": imad_ach / imad_peak,
                         "note": "algorithmic IMADs of the butterflies (3 per modmul) of the forward launch; "
                                 "peak = 152 SMs x 64 IMAD lanes x max SM clock"}
        if "tc" in results:
            tc_flops = 2 * 16 * N * (n1 + n2) * rows   # 2 GEMMs, 4 x 4 digit products, fused K'
            tc_tfs = tc_flops / (results["tc"]["fwd_ms"] / 1e3) / 1e12
            # the forward call is timed alone over a region of milliseconds: the burst peak applies
            peak_tc = peaks["bf16_tflops"]
            roof_tc = {"bound": "tensor", "achieved": tc_tfs, "peak": peak_tc, "unit": "TFLOP/s",
                       "frac": tc_tfs / peak_tc,
                       "peak_kind": peak_kind + " bf16 dense (burst); fp16 operands, same nominal rate",
                       "kernel": "tensor-core forward NTT call (2 tcgen05 GEMMs per chunk, Stage 1 fused "
                                 "into the first)",
                       "traffic": traffic_for("paper_2212_14191_gb300/csrc/ntt_tc.cu", "tc_fwd_call_n65536")}
        roof = roof_alu if head == "u32" else roof_tc
        line = {
            "metric": METRIC,
            "value": results[head]["kops"],
            "unit": "KOPS",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": total_head / args.steps * 1e3,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": "batched negacyclic NTT+INTT, N=2^16, %d RNS limbs (30-bit primes), "
                                   "%d polynomials (%d MiB); one op = one limb transform"
                                   % (NTT_LIMBS, NTT_BATCH, rows * N * 4 >> 20),
                       "path": head, "l2": ("inputs larger than L2 (%d MiB), no flush" if rows * N * 4 > 129e6 else
                              "inputs of %d MiB, which fit in L2; no flush") % (rows * N * 4 >> 20),
                       "parallelism": "replicas" if ws > 1 else "1 GPU"},
            "paths": results,
            "hmult": hm,
            "ops": ops,
            "heax_sets": heax_res,
            "mixed_batch": batch_res,
            "serving": serve_res,
            "roofline": roof,
            "roofline_u32": roof_u32,
            "roofline_u32_alu": roof_alu,
            "roofline_u32_imad": roof_imad,
            "roofline_tc": roof_tc,
            "e2e": {"value": ops_per_step * e2e_steps * ws / e2e_t / 1e3, "unit": "KOPS",
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
            "gpu_launches": launches_per_step[head] * args.steps,
            "clocks": clocks,
        }
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_oracle_kops()
            if not args.no_hmult:
                line["cpu_baseline"]["hmult_oracle"] = cpu_oracle_hmult()
        print(json.dumps(line))
    ctx.close()
    R.finish(ws)


def other_ops(args, fhe, hctx, a, b, evk, st, barrier, max_over_ranks, ws):
    """HROTATE (rotation by one slot; the relinearisation key stands in for the rotation key,
    which has the same layout), four hoisted rotations of the same ciphertexts (by 1, 2 and 3
    slots and the conjugation, one ModUp shared; one op = one rotated ciphertext), CMULT and
    HADD on the HMULT workload: 128 ciphertexts of 24 limbs at N = 2^16. CMULT and HADD are HBM
    streams; their fraction is of the measured HBM bandwidth."""
    import torch
    peaks, _ = measured_peaks()
    res = {"config": "N=2^16, 24 ciphertext limbs (+ 8 special primes for HROTATE), %d ciphertexts per call"
                     % args.hmult_batch}
    galois = 5                                   # 5^1 mod 2N: rotation of the slots by one
    pt = b[0]                                    # any (24, 128, N) residues serve as a plaintext
    out = torch.empty_like(a)
    rots = (5, 25, 125, 2 * N - 1)
    hout = torch.empty((len(rots),) + tuple(a.shape), dtype=a.dtype, device=a.device)
    limb_bytes = N * args.hmult_batch * 4
    cases = (("hrotate", lambda: hctx.hrotate(a, evk, LOGN, galois, out=out), None, args.hmult_steps, 1),
             ("hrotate_hoisted_x4", lambda: hctx.hrotate_hoisted(a, [evk] * len(rots), LOGN, rots, out=hout), None,
              args.hmult_steps, len(rots)),
             ("cmult", lambda: hctx.cmult(a, pt, LOGN, out=out), 5 * HM_LIMBS * limb_bytes, 10, 1),
             ("hadd", lambda: hctx.hadd(a, b, LOGN, out=out), 6 * HM_LIMBS * limb_bytes, 10, 1))
    for name, fn, nbytes, reps, nrot in cases:
        fn()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push(name)
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.nvtx.range_pop()
        barrier()
        t = max_over_ranks(e0.elapsed_time(e1) / 1e3) / reps
        res[name] = {"kops": nrot * args.hmult_batch * ws / t / 1e3, "ms_per_call": t * 1e3}
        if nrot > 1:
            res[name]["ms_per_rotation"] = t * 1e3 / nrot
            if "hrotate" in res:                 # single rotations per hoisted rotation time
                res[name]["speedup_vs_single"] = res["hrotate"]["ms_per_call"] / (t * 1e3 / nrot)
        if nbytes:
            res[name]["hbm_frac"] = nbytes / t / 1e9 / peaks["hbm_gbs"]
    fhe.fhe_device_status(hctx.handle, 1)
    del out, hout
    return res


# Table (HEAX comparison) parameter sets in 30-bit primes: log PQ / 30 rounded up, split
# into L ciphertext limbs and K special primes with P > Q (one key-switching slice, dnum = 1).
HEAX_SETS = tuple((h.name, h.logN, h.L, h.K) for h in CFG.HEAX_SETS)
HEAX_BATCH = CFG.HEAX_BATCH
HEAX_BATCH_SWEEP = CFG.HEAX_BATCH_SWEEP
PAPER_A100 = {"Set_A": (910134, 913267, 88048), "Set_B": (449974, 449084, 27564), "Set_C": (209337, 209178, 3825)}


def heax_sets(args, fhe, st, barrier, max_over_ranks, ws):
    """#NTT/s, #INTT/s (one op = one limb transform) and #HMULT/s (HMULT + relinearisation +
    rescale, one op = one ciphertext pair) at the paper's HEAX comparison sets, 1024
    ciphertexts per call, on the plain path with autotuned variants. The paper's A100 numbers
    are context, not targets. `batch_sweep` gives #NTT/s and #HMULT/s of each set at 32 to 1024
    ciphertexts per call (the batch-size study of Sec. VI-E), with the variants tuned at 1024."""
    import torch
    from paper_2212_14191_gb300 import inputs as I
    allp = fhe.fhe_gen_primes(16, 30, 16)
    res = {"config": "L ciphertext limbs + K special primes of 30 bits, dnum=1, %d ciphertexts per call" % HEAX_BATCH}

    def timed(fn, reps):
        for _ in range(3):
            fn()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / 1e3) / reps

    for name, logn, L, K in HEAX_SETS:
        n = 1 << logn
        ps, qs = allp[:K], allp[K:K + L]
        c = fhe.Context(logn, qs, ps, alpha=L, default_path=fhe.FHE_NTT_U32)
        rows_b = 4 * HEAX_BATCH                      # limb transforms: 4 limbs x batch polynomials
        x = fhe.to_device(I.uniform_residues(200 + logn, (qs + ps)[:4], HEAX_BATCH, n))   # L + K >= 4
        r = {"N": n, "L": L, "K": K}
        fhe.fhe_autotune_ntt(c.handle, logn, x.data_ptr(), 4, HEAX_BATCH, reps=2, stream=st.cuda_stream)
        for key, inv in (("ntt_per_s", False), ("intt_per_s", True)):
            fn = fhe.fhe_ntt_inv if inv else fhe.fhe_ntt_fwd
            for _ in range(3):
                fn(c.handle, fhe.FHE_NTT_U32, logn, x.data_ptr(), 0, 4, HEAX_BATCH, st.cuda_stream)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(20):
                fn(c.handle, fhe.FHE_NTT_U32, logn, x.data_ptr(), 0, 4, HEAX_BATCH, st.cuda_stream)
            e1.record(st)
            barrier()
            t = max_over_ranks(e0.elapsed_time(e1) / 1e3) / 20
            r[key] = rows_b * ws / t
        a = fhe.to_device(I.uniform_residues(210 + logn, qs, 2 * HEAX_BATCH, n)).view(L, 2, HEAX_BATCH, n) \
            .permute(1, 0, 2, 3).contiguous()
        b = fhe.to_device(I.uniform_residues(211 + logn, qs, 2 * HEAX_BATCH, n)).view(L, 2, HEAX_BATCH, n) \
            .permute(1, 0, 2, 3).contiguous()
        evk = fhe.to_device(I.uniform_residues(212 + logn, qs + ps, 2, n)).view(L + K, 1, 2, n) \
            .permute(1, 2, 0, 3).contiguous()
        out = torch.empty((2, L - 1, HEAX_BATCH, n), dtype=torch.int32, device="cuda")
        for _ in range(3):
            c.hmult(a, b, evk, logn, out=out)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(10):
            c.hmult(a, b, evk, logn, out=out)
        e1.record(st)
        barrier()
        t = max_over_ranks(e0.elapsed_time(e1) / 1e3) / 10
        r["hmult_per_s"] = HEAX_BATCH * ws / t
        r["paper_a100"] = dict(zip(("ntt_per_s", "intt_per_s", "hmult_per_s"), PAPER_A100[name]))
        sweep = {}
        for nb in HEAX_BATCH_SWEEP:
            if nb >= HEAX_BATCH:
                sweep[str(HEAX_BATCH)] = {"ntt_per_s": r["ntt_per_s"], "hmult_per_s": r["hmult_per_s"]}
                continue
            xs = x[:, :nb].contiguous()
            an, bn = a[:, :, :nb].contiguous(), b[:, :, :nb].contiguous()
            on = torch.empty((2, L - 1, nb, n), dtype=torch.int32, device="cuda")
            tn = timed(lambda: fhe.fhe_ntt_fwd(c.handle, fhe.FHE_NTT_U32, logn, xs.data_ptr(), 0, 4, nb,
                                               st.cuda_stream), 20)
            th = timed(lambda: c.hmult(an, bn, evk, logn, out=on), 10)
            sweep[str(nb)] = {"ntt_per_s": 4 * nb * ws / tn, "hmult_per_s": nb * ws / th}
            del xs, an, bn, on
        r["batch_sweep"] = sweep
        fhe.fhe_device_status(c.handle, 1)
        res[name] = r
        c.close()
        del a, b, evk, out, x
        torch.cuda.empty_cache()
    return res


def mixed_batch(args, fhe, ctx, qs, ps, st, barrier, max_over_ranks, ws):
    """Uneven batch: `--batch-ops` operations, kind uniform over {NTT, INTT, HMULT}, N uniform
    over {2^14, 2^15, 2^16}, level count (ciphertext limbs) uniform in 3..44, batch 1 each.
    One CUDA-graph replay of the persistent plan (one persistent launch popping every
    operation's stage tiles from a device queue) vs. the grouped plan (group after group) vs.
    one library call per operation."""
    import torch
    g = np.random.default_rng(4)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4)
    sh = st.cuda_stream
    n_ops = args.batch_ops
    mods = qs + ps
    dnum = -(-len(qs) // HM_ALPHA)
    evk = {}
    ops, tensors, desc = [], [], []
    limb_transforms = 0
    for i in range(n_ops):
        kind = int(g.integers(0, 3))
        logn = int(g.choice(list(CFG.MIXED_BATCH.logNs)))
        nl = int(g.integers(CFG.MIXED_BATCH.limb_range[0], CFG.MIXED_BATCH.limb_range[1] + 1))
        n = 1 << logn
        if kind < 2:
            d = torch.randint(0, 1 << 29, (nl, 1, n), dtype=torch.int32, device="cuda", generator=gen)
            k = fhe.FHE_OPK_NTT_FWD if kind == 0 else fhe.FHE_OPK_NTT_INV
            ops.append(fhe.FheOp(kind=k, logN=logn, first_limb=0, n_limbs=nl, batch=1, data=d.data_ptr()))
            tensors.append(d)
            desc.append((k, logn, nl, d))
            limb_transforms += nl
        else:
            if logn not in evk:
                evk[logn] = torch.randint(0, 1 << 29, (dnum, 2, len(mods), n), dtype=torch.int32, device="cuda",
                                          generator=gen)
            a = torch.randint(0, 1 << 29, (2, nl, 1, n), dtype=torch.int32, device="cuda", generator=gen)
            b = torch.randint(0, 1 << 29, (2, nl, 1, n), dtype=torch.int32, device="cuda", generator=gen)
            out = torch.empty((2, nl - 1, 1, n), dtype=torch.int32, device="cuda")
            ops.append(fhe.FheOp(kind=fhe.FHE_OPK_HMULT, logN=logn, n_limbs=nl, batch=1, a=a.data_ptr(),
                                 b=b.data_ptr(), evk=evk[logn].data_ptr(), out=out.data_ptr()))
            tensors += [a, b, out]
            desc.append((fhe.FHE_OPK_HMULT, logn, nl, (a, b, out)))
    plan = fhe.fhe_batch_create_ex(ctx.handle, ops, fhe.FHE_BATCH_PERSISTENT, 0)
    gplan = fhe.fhe_batch_create_ex(ctx.handle, ops, fhe.FHE_BATCH_GROUPED, 0)
    nbytes = max(fhe.fhe_batch_scratch_bytes(plan), fhe.fhe_batch_scratch_bytes(gplan))
    scratch = torch.empty(nbytes // 4 + 4, dtype=torch.int32, device="cuda")
    fhe.fhe_batch_capture(plan, scratch.data_ptr(), nbytes)
    fhe.fhe_batch_capture(gplan, scratch.data_ptr(), nbytes)
    per_op_bytes = max(fhe.fhe_scratch_bytes(ctx.handle, fhe.FHE_OP_HMULT, lg, 44, 1) for lg in (14, 15, 16))
    op_scratch = torch.empty(per_op_bytes // 4 + 4, dtype=torch.int32, device="cuda")

    def per_op():
        for k, logn, nl, t in desc:
            if k == fhe.FHE_OPK_NTT_FWD:
                fhe.fhe_ntt_fwd(ctx.handle, fhe.FHE_NTT_U32, logn, t.data_ptr(), 0, nl, 1, sh)
            elif k == fhe.FHE_OPK_NTT_INV:
                fhe.fhe_ntt_inv(ctx.handle, fhe.FHE_NTT_U32, logn, t.data_ptr(), 0, nl, 1, sh)
            else:
                a, b, out = t
                fhe.fhe_hmult(ctx.handle, logn, nl, 1, a.data_ptr(), b.data_ptr(), evk[logn].data_ptr(),
                              out.data_ptr(), op_scratch.data_ptr(), per_op_bytes, sh)

    def timed(fn, reps):
        fn()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / 1e3 / reps)

    t_graph = timed(lambda: fhe.fhe_batch_launch(plan, sh), 3)
    t_grouped = timed(lambda: fhe.fhe_batch_launch(gplan, sh), 3)
    t_ops = timed(per_op, 2)
    n_hm = sum(1 for d in desc if d[0] == fhe.FHE_OPK_HMULT)
    # every operation of both plans against its single call, after the timed regions: the
    # in-place NTT buffers are restored to one state before each run, the HMULT outputs cleared
    ntt_t = [t for k, _, _, t in desc if k != fhe.FHE_OPK_HMULT]
    hm_out = [t[2] for k, _, _, t in desc if k == fhe.FHE_OPK_HMULT]
    start = [t.clone() for t in ntt_t]

    def run_from_start(fn):
        torch.cuda.synchronize()
        for t, t0 in zip(ntt_t, start):
            t.copy_(t0)
        for o in hm_out:
            o.zero_()
        torch.cuda.synchronize()
        fn()
        torch.cuda.synchronize()
        return [t.clone() for t in ntt_t + hm_out]

    got_p = run_from_start(lambda: fhe.fhe_batch_launch(plan, sh))
    got_g = run_from_start(lambda: fhe.fhe_batch_launch(gplan, sh))
    want = run_from_start(per_op)
    bad_p = sum(1 for x, y in zip(got_p, want) if not torch.equal(x, y))
    bad_g = sum(1 for x, y in zip(got_g, want) if not torch.equal(x, y))
    del start, got_p, got_g, want
    assert bad_p == 0 and bad_g == 0, (bad_p, bad_g)
    res = {"ops": n_ops, "hmult_ops": n_hm, "ntt_ops": n_ops - n_hm, "ntt_limb_transforms": limb_transforms,
           "graph_ms": t_graph * 1e3, "grouped_graph_ms": t_grouped * 1e3, "per_op_ms": t_ops * 1e3,
           "graph_kops": n_ops * ws / t_graph / 1e3, "grouped_graph_kops": n_ops * ws / t_grouped / 1e3,
           "per_op_kops": n_ops * ws / t_ops / 1e3, "scratch_bytes": nbytes,
           "checked": {"ops": n_ops, "persistent_mismatches": bad_p, "grouped_mismatches": bad_g,
                       "against": "one library call per operation from the same inputs"},
           "config": "N in {2^14,2^15,2^16}, 3..44 limbs, batch 1 per op; graph replay of the persistent plan "
                     "(one launch, device work queue) vs the grouped plan vs one call per op",
           "ntt_variant_16": [fhe.fhe_ntt_get_variant(ctx.handle, 16, 0), fhe.fhe_ntt_get_variant(ctx.handle, 16, 1)]}
    fhe.fhe_device_status(ctx.handle, 1)
    fhe.fhe_batch_destroy(plan)
    fhe.fhe_batch_destroy(gplan)
    del tensors, scratch, op_scratch, evk
    torch.cuda.empty_cache()
    return res


def serving_bench(args, fhe, qs, ps):
    """Poisson streams of HMULT / RESCALE / KEYSWITCH requests, N in {2^15, 2^16}, 3..24 limbs,
    operands and evaluation keys resident in HBM, admitted by HBM footprint (24 GiB budget),
    continuous batching over 4 CUDA streams. Two steady-state runs of `--serving-seconds` of
    arrivals each: the configured mean rate (50k requests/s, above capacity; a request not
    admitted within 50 ms of its arrival is rejected), whose completion rate is the sustainable
    capacity, then 0.8x that capacity (nothing rejected). Operands come from a pool of two
    operand sets per (operation, N, limbs), since requests only read them; results are dropped
    as batches complete."""
    import torch
    from paper_2212_14191_gb300 import serving as S
    sv = CFG.SERVING
    logns = sv.logNs
    ctxs = {lg: fhe.Context(lg, qs[:HM_LIMBS], ps, alpha=HM_ALPHA) for lg in logns}
    dnum = -(-HM_LIMBS // HM_ALPHA)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    evks = {lg: torch.randint(0, 1 << 29, (dnum, 2, HM_LIMBS + HM_K, 1 << lg), dtype=torch.int32, device="cuda",
                              generator=gen) for lg in logns}
    pool = {}

    def make_inputs(kind, logN, nl, rid):
        key = (kind, logN, nl, rid % 2)
        if key not in pool:
            n = 1 << logN
            if kind == S.KEYSWITCH:
                pool[key] = (torch.randint(0, 1 << 29, (nl, 1, n), dtype=torch.int32, device="cuda", generator=gen),)
            else:
                k = 2 if kind == S.HMULT else 1
                pool[key] = tuple(torch.randint(0, 1 << 29, (2, nl, 1, n), dtype=torch.int32, device="cuda",
                                                generator=gen) for _ in range(k))
        return pool[key]

    kinds = [S.HMULT, S.RESCALE, S.KEYSWITCH]

    def run(rate, seconds, seed, admit_timeout_s):
        n = max(1, int(rate * seconds))
        reqs = S.poisson_requests(seed, n, rate, kinds, logns, sv.limb_range, make_inputs)
        server = S.Server(ctxs, evks, budget_bytes=sv.budget_bytes, n_streams=sv.streams, max_batch=sv.max_batch,
                          admit_timeout_s=admit_timeout_s, keep_results=False)
        torch.cuda.synchronize()
        st = server.run(reqs)
        torch.cuda.synchronize()
        st["offered_req_s"] = rate
        st["arrival_s"] = reqs[-1].arrival
        st["completed_req_s"] = st["completed"] / st["wall_s"]
        return st

    run(sv.rate_per_s, 0.05, 6, 0.05)                      # warm-up (pool, allocator, kernels)
    over = run(sv.rate_per_s, args.serving_seconds, 7, 0.05)
    capacity = over["completed_req_s"]
    steady = run(0.8 * capacity, args.serving_seconds, 8, None)
    for c in ctxs.values():
        fhe.fhe_device_status(c.handle, 1)
        c.close()
    del pool, evks
    torch.cuda.empty_cache()
    return {"overload": over, "steady_0p8": steady, "capacity_req_s": capacity,
            "config": ("Poisson arrivals for %.1f s each: %d req/s (rejection after 50 ms without admission) and "
                       "0.8 x the measured capacity; HMULT/RESCALE/KEYSWITCH, N in {2^15,2^16}, 3..24 limbs, "
                       "24 GiB admission budget, 4 streams, batches of <= 32" % (args.serving_seconds, sv.rate_per_s))}


def main():
    global NTT_BATCH
    args = parse()
    NTT_BATCH = args.ntt_batch
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
