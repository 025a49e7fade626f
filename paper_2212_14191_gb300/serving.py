"""Continuous-batching request loop for HMULT / RESCALE / KEYSWITCH (the API layer of
Sec. IV-E: it collects operation requests, picks batch sizes from the hardware's memory and
invokes the kernels, with intermediate results kept in device memory).

Each request names an operation, a ring degree N = 2^logN and a limb count, and its
ciphertext operands already live in HBM; evaluation keys are resident per ring degree.
Operands may still be in production on the stream that is current when `run` is called:
every launch stream first waits for an event recorded on that stream at the start of the
run, so no batch reads an operand before it is written.
The server
  * admits a request only while the HBM footprint of everything admitted and in flight
    (operands, result and the batch's scratch share) stays under `budget_bytes`;
  * keeps one queue per (operation, N, limbs) class and, whenever one of its CUDA streams is
    free, launches up to `max_batch` queued requests of the class with the oldest request as
    one batched library call on that stream;
  * polls completion events, releases the footprint and records latencies;
  * under overload, optionally rejects a request that has waited for admission longer than
    `admit_timeout_s` while the budget was full (it is marked rejected and never launched);
  * detects failures on the host: if batches are in flight and none completes for `stall_s`
    seconds the run stops with an error naming them, and after the run every context's
    device error word is read (fhe_device_status), so an expired bounded wait inside a
    kernel (whose results are then incomplete) is reported instead of returned.
Requests that arrive while others run are admitted as memory frees and join the next
batches (continuous batching); batches on different streams overlap on the GPU.
All arithmetic runs in libfhe's kernels; batching changes only the batch dimension, so a
request's result is identical alone and in any mix.
"""
import collections
import time

import torch

from . import fhe

HMULT, RESCALE, KEYSWITCH = "hmult", "rescale", "keyswitch"


class Request:
    __slots__ = ("rid", "kind", "logN", "nl", "arrival", "inputs", "out", "t_admit", "t_launch", "t_done",
                 "footprint", "rejected")

    def __init__(self, rid, kind, logN, nl, arrival, inputs):
        self.rid, self.kind, self.logN, self.nl, self.arrival = rid, kind, logN, nl, arrival
        self.inputs = inputs  # HMULT: (a, b) each (2, nl, 1, N); RESCALE: (ct,); KEYSWITCH: (d2,) (nl, 1, N)
        self.out = None
        self.t_admit = self.t_launch = self.t_done = None
        self.footprint = 0
        self.rejected = False


def _out_shape(kind, nl, batch, n):
    if kind == HMULT or kind == RESCALE:
        return (2, nl - 1, batch, n)
    return (2, nl, batch, n)


def _op_code(kind):
    return {HMULT: fhe.FHE_OP_HMULT, RESCALE: fhe.FHE_OP_RESCALE, KEYSWITCH: fhe.FHE_OP_KEYSWITCH}[kind]


class Server:
    def __init__(self, contexts, evks, budget_bytes, n_streams=4, max_batch=16, stall_s=60.0,
                 admit_timeout_s=None, keep_results=True):
        """contexts: {logN: fhe.Context}; evks: {logN: int32 CUDA tensor (dnum, 2, nq+np, N)}.
        admit_timeout_s: None waits for memory indefinitely; otherwise a request that cannot be
        admitted within this many seconds of its arrival is rejected.
        keep_results: False drops each batch's output once it completes (r.out stays None), for
        long load measurements whose results are not read."""
        self.ctx = contexts
        self.evk = evks
        self.budget = budget_bytes
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.max_batch = max_batch
        self.stall_s = stall_s
        self.admit_timeout_s = admit_timeout_s
        self.keep_results = keep_results
        self._ready = None   # event on the caller's stream at the start of run()

    def check_device(self):
        """Raise fhe.FheError if a kernel of any context reported an expired bounded wait."""
        for ctx in self.ctx.values():
            fhe.fhe_device_status(ctx.handle, 1)

    def footprint(self, r):
        """Bytes a request holds while admitted: its operands, the gathered copy of them that
        its batch makes, its result and its share of the batch's scratch. The result stays
        allocated after completion (it belongs to the caller) and is no longer counted then."""
        n = 1 << r.logN
        ins = 2 * sum(t.numel() * 4 for t in r.inputs)   # the operands and their gathered copy
        out = 4 * n
        for d in _out_shape(r.kind, r.nl, 1, n)[:-1]:
            out *= d
        scratch = fhe.fhe_scratch_bytes(self.ctx[r.logN].handle, _op_code(r.kind), r.logN, r.nl, 1)
        return ins + out + scratch

    def _producer_event(self):
        """An event on the caller's current stream: everything queued there so far (the
        operands' producers included) completes before any batch of this run starts."""
        ev = torch.cuda.Event()
        ev.record(torch.cuda.current_stream())
        return ev

    def _launch(self, reqs, stream):
        r0 = reqs[0]
        kind, logN, nl, n = r0.kind, r0.logN, r0.nl, 1 << r0.logN
        ctx = self.ctx[logN]
        bsz = len(reqs)
        if self._ready is not None:
            stream.wait_event(self._ready)   # operands written on the producer stream come first
        with torch.cuda.stream(stream):
            if kind == KEYSWITCH:
                ins = [torch.cat([r.inputs[0] for r in reqs], dim=1)]
            else:
                ins = [torch.cat([r.inputs[k] for r in reqs], dim=2) for k in range(len(r0.inputs))]
            out = torch.empty(_out_shape(kind, nl, bsz, n), dtype=torch.int32, device="cuda")
            nbytes = fhe.fhe_scratch_bytes(ctx.handle, _op_code(kind), logN, nl, bsz)
            scratch = torch.empty(max(4, nbytes // 4 + 4), dtype=torch.int32, device="cuda")
            sh = stream.cuda_stream
            if kind == HMULT:
                fhe.fhe_hmult(ctx.handle, logN, nl, bsz, ins[0].data_ptr(), ins[1].data_ptr(),
                              self.evk[logN].data_ptr(), out.data_ptr(), scratch.data_ptr(), nbytes, sh)
            elif kind == RESCALE:
                fhe.fhe_rescale(ctx.handle, logN, nl, bsz, ins[0].data_ptr(), out.data_ptr(), scratch.data_ptr(),
                                nbytes, sh)
            else:
                fhe.fhe_keyswitch(ctx.handle, logN, nl, bsz, ins[0].data_ptr(), self.evk[logN].data_ptr(),
                                  out.data_ptr(), scratch.data_ptr(), nbytes, sh)
            ev = torch.cuda.Event()
            ev.record(stream)
        if self.keep_results:
            for j, r in enumerate(reqs):
                r.out = out[:, :, j:j + 1]
        return {"reqs": reqs, "event": ev, "keep": (ins, out, scratch), "stream": stream}

    def run(self, requests, clock=time.perf_counter):
        """Serve `requests` (sorted by arrival, seconds from start) to completion or rejection.

        Returns a dict of latency percentiles (ms) over the completed requests, throughput,
        batch statistics and the number rejected.
        """
        self._ready = self._producer_event()
        pending = collections.OrderedDict()   # class -> deque of admitted requests
        arrivals = collections.deque(requests)
        inflight = []
        used = 0
        free_streams = list(self.streams)
        batches = []
        peak_used = 0
        t0 = clock()
        done = 0
        rejected = 0
        n = len(requests)
        last_progress = 0.0
        while done < n:
            now = clock() - t0
            if inflight and now - last_progress > self.stall_s:
                stuck = sorted({(b["reqs"][0].kind, b["reqs"][0].logN, b["reqs"][0].nl) for b in inflight})
                raise RuntimeError("serving: no batch completed for %.1f s; in flight: %s" % (now - last_progress, stuck))
            # admission by HBM footprint
            while arrivals and arrivals[0].arrival <= now:
                r = arrivals[0]
                if not r.footprint:
                    r.footprint = self.footprint(r)
                if used + r.footprint > self.budget and (inflight or any(pending.values())):
                    if self.admit_timeout_s is not None and now - r.arrival > self.admit_timeout_s:
                        arrivals.popleft()
                        r.rejected = True
                        rejected += 1
                        done += 1
                        continue
                    break
                arrivals.popleft()
                r.t_admit = now
                used += r.footprint
                peak_used = max(peak_used, used)
                pending.setdefault((r.kind, r.logN, r.nl), collections.deque()).append(r)
            # launch on free streams, oldest class first
            while free_streams:
                live = [(q[0].t_admit, key) for key, q in pending.items() if q]
                if not live:
                    break
                _, key = min(live)
                q = pending[key]
                reqs = [q.popleft() for _ in range(min(self.max_batch, len(q)))]
                for r in reqs:
                    r.t_launch = now
                if not inflight:
                    last_progress = now
                inflight.append(self._launch(reqs, free_streams.pop()))
                batches.append(len(reqs))
            # completions
            still = []
            for b in inflight:
                if b["event"].query():
                    t = clock() - t0
                    for r in b["reqs"]:
                        r.t_done = t
                        used -= r.footprint
                    done += len(b["reqs"])
                    free_streams.append(b["stream"])
                    last_progress = t
                else:
                    still.append(b)
            inflight = still
        self.check_device()
        served = [r for r in requests if not r.rejected]
        t_end = max((r.t_done for r in served), default=clock() - t0)
        lat = sorted((r.t_done - r.arrival) * 1e3 for r in served) or [0.0]

        def pct(p):
            return lat[min(len(lat) - 1, int(round(p / 100.0 * (len(lat) - 1))))]

        return {"requests": n, "completed": len(served), "rejected": rejected,
                "p50_ms": pct(50), "p99_ms": pct(99), "max_ms": lat[-1],
                "throughput_kops": len(served) / t_end / 1e3, "wall_s": t_end, "batches": len(batches),
                "mean_batch": sum(batches) / max(1, len(batches)), "peak_footprint_bytes": peak_used,
                "budget_bytes": self.budget, "streams": len(self.streams)}


def poisson_requests(seed, n, rate_per_s, kinds, logNs, nl_range, make_inputs):
    """n requests with exponential inter-arrival times (mean 1/rate); kind, ring degree and
    limb count drawn uniformly. make_inputs(kind, logN, nl, rid) returns the operand tensors."""
    import numpy as np
    g = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(n):
        t += g.exponential(1.0 / rate_per_s)
        kind = kinds[int(g.integers(0, len(kinds)))]
        logN = int(logNs[int(g.integers(0, len(logNs)))])
        nl = int(g.integers(nl_range[0], nl_range[1] + 1))
        out.append(Request(rid, kind, logN, nl, t, make_inputs(kind, logN, nl, rid)))
    return out
