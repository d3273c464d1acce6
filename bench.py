"""Benchmark: HE rotations/sec at N=2^16 (batched rotation workload).

Workload (one "step"): 256 CKKS ciphertexts at N = 2^16 over 24 x 50-bit Q
limbs + 4 x 60-bit P limbs, dnum 6, each at a level ~ U{4..24}, each rotated
by its own amount ~ U[1, 2^15) with its own resident rotation key (one key per
distinct amount, ~45 GB of keys), all in one fheon_rotate_batch call.  Inputs
are fresh encryptions of U[-1, 1] slot vectors (synthetic, seeded).  Keys and
ciphertexts (> 45 GB) exceed the 129 MB L2, so no flush is needed.

Arms:
  default          the CUDA library; prints one JSON line with roofline,
                   cpu_baseline, e2e, clocks, gpu_launches.
  --impl reference the CPU oracle (test infrastructure) timed on this host's
                   cores on a bounded sample of the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2510_03996_gb300 import synth  # noqa: E402

METRIC = "HE rotations/sec at N=2^16"
UNIT = "rotations/s"
WORKLOAD = "rot_n16"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# DRAM bytes the kernel moved per launch over its minimum traffic (sources read
# once, results written once), from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the 16-ciphertext case of this workload; a full
# launch's traffic is this ratio times its own minimum bytes.
TRAFFIC_OVER_MIN = {"up_bconv_ntt_cols": 902.6 / 895.5}


def algorithmic_costs(N, L, K, alpha, level, q_lazy=True, p_lazy=False):
    """Algorithmic work of one rotation at `level`, in total and per kernel.

    bytes: what must cross HBM at least once (key + ciphertext in and out).
    Per kernel: 'mm' = 64-bit modular products by kind (one per NTT butterfly
    -- forward 'ct' or inverse 'gs', 'lazy' on primes below 2^54 (q_lazy for
    the Q primes, p_lazy for the P primes) else 'harvey' -- and one 'mac' per
    base-conversion multiply-accumulate), or 'bytes' for the streaming key
    inner product.  Pass A of a size-N transform covers log2(N)/2 stages
    (floor), pass B the rest."""
    beta = (level + alpha - 1) // alpha
    limb = 8 * N
    logN = N.bit_length() - 1
    b1, b2 = logN // 2, logN - logN // 2
    half = N // 2
    qk, pk = ("lazy" if q_lazy else "harvey"), ("lazy" if p_lazy else "harvey")
    key_bytes = 2 * beta * (level + K) * limb
    ct_bytes = 4 * level * limb  # read (c0, c1), write (c0', c1')
    new_q = beta * level - level  # raised Q limbs (every digit's other Q limbs)
    new_p = beta * K              # raised P limbs
    new_limbs = new_q + new_p
    digits = [min(alpha, level - j * alpha) for j in range(beta)]
    modup_macs = N * sum(d * (level + K - d) for d in digits)

    def mm(**kw):
        return {k: v for k, v in kw.items() if v}

    k = {
        "ic_intt_rows": {"mm": mm(**{"gs_" + qk: level * half * b2})},
        "ic_intt_cols": {"mm": mm(**{"gs_" + qk: level * half * b1})},
        # both prime-class launches read every source limb
        "up_bconv_ntt_cols": {"mm": mm(**{"ct_" + qk: new_q * half * b1}, **{"ct_" + pk: new_p * half * b1},
                                       mac=modup_macs) if qk != pk else
                              mm(**{"ct_" + qk: new_limbs * half * b1}, mac=modup_macs),
                              "min_bytes": (2 * level + new_limbs) * limb},
        "up_ntt_rows": {"mm": mm(**{"ct_" + qk: new_q * half * b2}, **{"ct_" + pk: new_p * half * b2})
                        if qk != pk else mm(**{"ct_" + qk: new_limbs * half * b2})},
        "ks_inner": {"bytes": key_bytes + beta * (level + K) * limb + 2 * (level + K) * limb,
                     "min_bytes": key_bytes + beta * (level + K) * limb + 2 * (level + K) * limb},
        "dn_intt_rows": {"mm": mm(**{"gs_" + pk: 2 * K * half * b2})},
        "dn_intt_cols": {"mm": mm(**{"gs_" + pk: 2 * K * half * b1})},
        "dn_bconv_ntt_cols": {"mm": mm(**{"ct_" + qk: 2 * level * half * b1}, mac=2 * level * K * N)},
        "dn_ntt_rows_combine": {"mm": mm(**{"ct_" + qk: 2 * level * half * b2})},
    }
    return dict(bytes=key_bytes + ct_bytes, kernels=k)


def rooflines(prof, costs, steps, hbm_peak, alu_rates):
    """Per-kernel achieved rate against its roofline.  The inner product: GB/s
    against hbm_peak.  ALU kernels: their modular products by kind; the
    shortest time they can take is sum_kind n_kind / rate_kind at the
    measured rates (alu_rates, steps/s), so frac = that time / the measured
    time, achieved = products / measured time and peak = products / shortest
    time, both in T modular products/s."""
    out = {}
    for name, (n, ms) in prof.items():
        if ms <= 0:
            continue
        work = [c["kernels"].get(name, {}) for c in costs]
        if any("bytes" in w for w in work):
            a = sum(w.get("bytes", 0) for w in work) * steps / (ms / 1e3) / 1e9
            out[name] = {"bound": "hbm", "achieved": a, "peak": hbm_peak, "unit": "GB/s", "frac": a / hbm_peak}
        elif any("mm" in w for w in work):
            tot = {}
            for w in work:
                for kind, v in w.get("mm", {}).items():
                    tot[kind] = tot.get(kind, 0) + v * steps
            prods = sum(tot.values())
            t_min = sum(v / alu_rates[kind] for kind, v in tot.items())
            a = prods / (ms / 1e3) / 1e12
            peak = prods / t_min / 1e12
            out[name] = {"bound": "alu", "achieved": a, "peak": peak, "unit": "Tmodmul/s", "frac": a / peak,
                         "mix": {k: round(v / prods, 4) for k, v in sorted(tot.items())}}
        out.get(name, {}).update({"launches": n, "avg_launch_ms": ms / n})
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "sm_min_mhz": float(min(sm)) if sm else None}


def step_summary(ms):
    """Median and largest of the intervals (ms) between consecutive steps'
    completions, and the step whose completion the largest one ends at."""
    if not ms:
        return {}
    k = int(np.argmax(ms))
    return {"step_ms_median": round(float(np.median(ms)), 3), "step_ms_max": round(float(ms[k]), 3),
            "slowest_step": k + 1}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def barrier_max(value, world, device="cuda"):
    """The maximum of `value` over the ranks (the slowest replica's time)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank, seconds, world, device="cuda"):
    """Whole-job rate of `world` independent replicas that each processed
    `units_per_rank` units: all units over the slowest replica's time."""
    return world * units_per_rank / barrier_max(seconds, world, device)


# ------------------------------------------------------------------ oracle timing
class OracleRunner:
    """The CPU oracle (single thread) set up once on the workload's parameters.
    One rotation key serves every sample: the work does not depend on which key."""

    def __init__(self, P, step):
        import oracle.ckks as O
        N = 1 << P["logN"]
        L = len(P["qbits"])
        mods = O.gen_primes(N, P["qbits"] + P["pbits"])
        self.oc = O.Ctx(N, mods[:L], mods[L:], P["dnum"], P["seed"])
        _, se = self.oc.keygen_sk()
        pk = self.oc.keygen_pk(se)
        self.g = O.galois_elt(step, N)
        self.key = self.oc.rotkey(se, self.g)
        self.ct = self.oc.encrypt(pk, synth.small_int_poly(P["seed"], 5, N, 1 << 40), 1)

    def rotate_seconds(self, level):
        c = self.oc.drop_level(self.ct, level)
        t0 = time.perf_counter()
        self.oc.rotate(c, self.g, self.key)
        return time.perf_counter() - t0

    def rate(self, levels, budget_s):
        done, t_total, used = 0, 0.0, []
        for lv in levels:
            t_total += self.rotate_seconds(lv)
            done += 1
            used.append(lv)
            if t_total > budget_s:
                break
        return done / t_total, done, t_total, used


def _oracle_worker(P, step, levels, barrier, results):
    """One host core's share of the all-cores oracle timing (a spawned process:
    no CUDA state is inherited)."""
    runner = OracleRunner(P, step)
    barrier.wait()
    t = sum(runner.rotate_seconds(lv) for lv in levels)
    results.put((len(levels), t))


def oracle_all_cores(P, step, levels, per_core=1, cores=None):
    """The oracle on every host core at once: one process per core, each with
    its own context and key, released together; each rotates `per_core` of
    the workload's items.  Rate = all rotations / the slowest process's time."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier, results = ctx.Barrier(cores), ctx.Queue()
    procs = []
    for c in range(cores):
        lv = [levels[(c * per_core + k) % len(levels)] for k in range(per_core)]
        p = ctx.Process(target=_oracle_worker, args=(P, step, lv, barrier, results))
        p.start()
        procs.append(p)
    out = [results.get() for _ in procs]
    for p in procs:
        p.join()
    done = sum(n for n, _ in out)
    slowest = max(t for _, t in out)
    return done / slowest, done, slowest, cores


def _oracle_server(P, step, cmd, results):
    """A reference-arm worker (a spawned process): rotates one ciphertext at
    each level it is sent, reports the seconds; None ends it."""
    runner = OracleRunner(P, step)
    results.put(("ready", 0.0))
    while True:
        lv = cmd.get()
        if lv is None:
            return
        results.put(("done", runner.rotate_seconds(lv)))


class OraclePool:
    """The oracle on every host core: one spawned process per core, each with
    its own context and key; a step sends one level to every process and
    lasts as long as the slowest."""

    def __init__(self, P, step, cores=None):
        import multiprocessing as mp
        self.cores = cores or os.cpu_count() or 1
        ctx = mp.get_context("spawn")
        self.results = ctx.Queue()
        self.cmds = [ctx.Queue() for _ in range(self.cores)]
        self.procs = [ctx.Process(target=_oracle_server, args=(P, step, q, self.results)) for q in self.cmds]
        for p in self.procs:
            p.start()
        for _ in self.procs:
            self.results.get()

    def step(self, levels):
        for q, lv in zip(self.cmds, levels):
            q.put(lv)
        return max(self.results.get()[1] for _ in levels)

    def close(self):
        for q in self.cmds:
            q.put(None)
        for p in self.procs:
            p.join()


def run_reference(args, rank, world):
    if rank != 0:
        return
    P = synth.params(WORKLOAD)
    levels, steps = synth.rotation_workload(P["seed"])
    pool = OraclePool(P, steps[0])
    n = pool.cores
    # each step rotates the next `cores` workload items, one per host core, at once
    item = 0

    def next_levels():
        nonlocal item
        lv = [levels[(item + c) % len(levels)] for c in range(n)]
        item += n
        return lv

    for _ in range(args.warmup):
        pool.step(next_levels())
    t_steps, per_step = [], []
    for _ in range(args.steps):
        lv = next_levels()
        t_steps.append(pool.step(lv))
        per_step.append(lv)
    pool.close()
    value = n * len(t_steps) / sum(t_steps)
    ms = 1e3 * sum(t_steps) / len(t_steps)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "batched rotation, N=2^16, 24x50-bit Q + 4x60-bit P, dnum 6, levels U{4..24}, "
                                   "steps U[1,2^15); a reference step rotates %d ciphertexts, one per host core" % n,
                       "levels_sampled": per_step, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": n, "kind": "oracle",
                             "sample": "%d rotations per step, one per host core at once, at the workload's item "
                                       "levels" % n},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ CUDA arm
def per_ciphertext_rate(ctx, ins, outs, steps, stream, reps=2):
    """The same rotations issued one ciphertext per call (fheon_rotate), the
    comparison point for the batched call."""
    import torch
    for c, o, r in zip(ins, outs, steps):
        ctx.rotate(c, r, o)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        for c, o, r in zip(ins, outs, steps):
            ctx.rotate(c, r, o)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"value": reps * len(ins) / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / reps}


def release(*ctxs):
    """Close contexts and hand their device memory back: torch's caching
    allocator keeps freed blocks per stream, and every context here has a
    stream of its own."""
    import torch
    for c in ctxs:
        c.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def lenet_timing(F, batch=32):
    """LeNet-5 encrypted inference (N = 2^15, 44 levels, no bootstrapping) over a
    batch of synthetic 1x28x28 U[0,1] inputs with random-init weights: seconds
    per inference (CUDA events around the batch), and the largest distance of
    the decrypted logits from the FP64 network with exact ReLUs."""
    import torch
    from paper_2510_03996_gb300 import lenet
    P = synth.params("lenet_n15")
    N = 1 << P["logN"]
    s = torch.cuda.Stream()
    ctx = F.Context(N, qbits=P["qbits"], pbits=P["pbits"], dnum=P["dnum"], scale=P["scale"], seed=P["seed"],
                    stream=s.cuda_stream)
    w = lenet.weights(P["seed"])
    xs = [synth.image(P["seed"], 700 + i, (1, 28, 28)) for i in range(batch)]
    betas = lenet.relu_bounds(xs, w)
    sk, pk = ctx.keygen()
    ctx.relinkeygen(sk)
    net = lenet.EncryptedLeNet(ctx, w, betas, ctx.L, P["scale"])
    ctx.rotkeygen(sk, net.rotation_steps())
    cts = [ctx.encrypt(pk, ctx.encode(lenet.pack_input(X, N // 2), ctx.L, P["scale"]), nonce=i)
           for i, X in enumerate(xs)]
    net.forward(cts[0])  # warm-up: working ciphertexts, plans
    net.forward_graph(cts[0])  # capture
    ctx.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    outs = [net.forward(ct) for ct in cts]
    e1.record(s)
    torch.cuda.synchronize()
    eager_secs = e0.elapsed_time(e1) / 1e3
    e0.record(s)
    gouts = [net.forward_graph(ct) for ct in cts]
    e1.record(s)
    torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    same = all(np.array_equal(ctx.ct_download(a), ctx.ct_download(b)) for a, b in zip(outs[:2], gouts[:2]))
    # the batch through batched layer applications (every layer over 8 inputs
    # per call: their rotations, products and series share launches)
    chunk = 8
    net.forward_batch(cts[:chunk])  # warm-up: the batch's working sets and plans
    ctx.sync()
    e0.record(s)
    bouts = []
    for i in range(0, batch, chunk):
        bouts += net.forward_batch(cts[i:i + chunk])
    e1.record(s)
    torch.cuda.synchronize()
    batched_secs = e0.elapsed_time(e1) / 1e3
    batch_same = all(np.array_equal(ctx.ct_download(a), ctx.ct_download(b)) for a, b in zip(outs[:2], bouts[:2]))
    err = 0.0
    for X, y in zip(xs, outs):
        got = np.asarray(ctx.decode(ctx.decrypt(sk, y))).real[:10]
        err = max(err, float(np.max(np.abs(got - lenet.forward_fp64(X, w)))))
    nkeys, kbytes = ctx.key_stats()
    del outs, gouts, bouts, cts, net, sk, pk
    release(ctx)
    return {"s_per_inference": min(secs, batched_secs) / batch, "graph_s_per_inference": secs / batch,
            "batched_s_per_inference": batched_secs / batch, "batched_chunk": chunk,
            "batched_equals_one_by_one": batch_same, "eager_s_per_inference": eager_secs / batch,
            "graph_equals_eager": same, "batch": batch, "keys": nkeys, "key_bytes": kbytes,
            "max_abs_logit_vs_fp64_exact_relu": err, "relu_bounds": betas, "levels": len(P["qbits"])}


def resnet_timing(F, n_inputs=2):
    """ResNet-20 encrypted inference with bootstrapping (N = 2^16, 37 primes:
    q_0, 16 levels of layers, 20 of bootstrapping) on synthetic 3x32x32 N(0,1)
    inputs with random-init weights: seconds per inference (CUDA events around
    the inputs, one after another), one bootstrap alone, and the decrypted
    logits against the FP64 network with exact ReLUs."""
    import torch
    from paper_2510_03996_gb300 import resnet
    P = synth.params("resnet_n16")
    N = 1 << P["logN"]
    s = torch.cuda.Stream()
    ctx = F.Context(N, qbits=P["qbits"], pbits=P["pbits"], dnum=P["dnum"], scale=P["scale"], seed=P["seed"],
                    stream=s.cuda_stream)
    w = resnet.weights(P["seed"])
    xs = [synth.image(P["seed"], 800 + i, (3, 32, 32), dist="normal") for i in range(n_inputs)]
    betas = resnet.relu_bounds(xs, w)
    sk, pk = ctx.keygen()
    t0 = time.time()
    net = resnet.EncryptedResNet(ctx, w, betas, P["scale"])
    net.keygen(sk)
    ctx.sync()
    t_prep = time.time() - t0
    cts = [ctx.drop_level(ctx.encrypt(pk, ctx.encode(resnet.pack_input(X, N // 2), ctx.L, P["scale"]), nonce=i),
                          net.in_level) for i, X in enumerate(xs)]
    net.forward(cts[0])  # warm-up: working ciphertexts, plans, workspace
    net.forward_graph(cts[0])  # capture
    ctx.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    outs = [net.forward(ct) for ct in cts]
    e1.record(s)
    torch.cuda.synchronize()
    eager_secs = e0.elapsed_time(e1) / 1e3
    e0.record(s)
    gouts = [net.forward_graph(ct) for ct in cts]
    e1.record(s)
    torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    same = all(np.array_equal(ctx.ct_download(a), ctx.ct_download(b)) for a, b in zip(outs, gouts))
    # the inputs as one batch: every layer and bootstrap over both at once
    net.forward_batch(cts)  # warm-up: the batch's working sets
    ctx.sync()
    e0.record(s)
    bouts = net.forward_batch(cts)
    e1.record(s)
    torch.cuda.synchronize()
    batch_secs = e0.elapsed_time(e1) / 1e3
    batch_same = all(np.array_equal(ctx.ct_download(a), ctx.ct_download(b)) for a, b in zip(outs, bouts))
    del bouts
    # one bootstrap alone: the sparse one (slots [0, N/4), one EvalMod) the
    # network mostly uses, and the full one
    z = ctx.drop_level(cts[0], 2)
    boot_ms_by = {}
    for (slots, unmasked), layer in sorted(net._boots.items()):
        ctx.layer_apply(layer, z)
        e0.record(s)
        for _ in range(5):
            ctx.layer_apply(layer, z)
        e1.record(s)
        torch.cuda.synchronize()
        name = ("sparse_%d_slots" % slots + ("_unmasked" if unmasked else "")) if slots else "full"
        boot_ms_by[name] = e0.elapsed_time(e1) / 5
    boot_ms = boot_ms_by.get("sparse_%d_slots" % (N // 4), boot_ms_by.get("full"))
    # one bootstrap launch by launch (events on the context's stream): share of each kernel
    ctx.profile_begin()
    ctx.layer_apply(net.boot, z)
    bprof = ctx.profile_end()
    btot = sum(v[1] for v in bprof.values())
    boot_kernels = {k: {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / btot, 4)}
                    for k, v in sorted(bprof.items(), key=lambda kv: -kv[1][1])[:12]}
    # where one inference spends its time: CUDA events around every step of
    # the plan (eager), summed by kind of step
    kind_ms = {}
    reg = {"x": cts[0]}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(net.plan) + 1)]
    ev[0].record(s)
    names = []
    for k, op in enumerate(net.plan):
        if op[0] == "layer":
            layer = op[1]
            name = next((n for n, l in net.layers.items() if l is layer), None)
            name = "relu" if name is None else ("conv" if "conv" in name or name.startswith("s") else name)
            reg[op[3]] = ctx.layer_apply(layer, reg[op[2]])
        elif op[0] == "scale":
            name = "shortcut_scale"
            reg[op[3]] = ctx.mul_const_rescale(reg[op[2]], op[1], net.scale)
        elif op[0] == "add":
            name = "add"
            A, Bc = (ctx.drop_level(reg[x], op[1]) if ctx.ct_info(reg[x])[0] > op[1] else reg[x] for x in (op[2], op[3]))
            reg[op[4]] = ctx.add(A, Bc)
        else:
            name = "bootstrap"
            reg[op[1]] = ctx.layer_apply(op[2], reg[op[1]])
        ev[k + 1].record(s)
        names.append(name)
    torch.cuda.synchronize()
    for k, name in enumerate(names):
        kind_ms[name] = kind_ms.get(name, 0.0) + ev[k].elapsed_time(ev[k + 1])
    del reg
    # the plain one-ciphertext-per-launch path: every rotation and product of
    # the same network through its own launch sequence, nothing hoisted
    ctx.set_batching(False)
    net.forward(cts[0])  # warm-up of the plain path's workspace
    ctx.sync()
    e0.record(s)
    for ct in cts:
        net.forward(ct)
    e1.record(s)
    torch.cuda.synchronize()
    plain_secs = e0.elapsed_time(e1) / 1e3
    ctx.set_batching(True)
    coeffs = [F.relu_coeffs(b, resnet.RELU_DEGREE) for b in betas]

    def cheb_relu(v, i):
        # the encrypted network's ReLU, the Chebyshev series at v / beta, in FP64
        z = v / betas[i]
        t0, t1 = np.ones_like(z), z
        y = coeffs[i][0] * t0 + coeffs[i][1] * t1
        for c in coeffs[i][2:]:
            t0, t1 = t1, 2.0 * z * t1 - t0
            y = y + c * t1
        return y
    err, err_cheb, agree = 0.0, 0.0, 0
    for X, y in zip(xs, outs):
        got = np.asarray(ctx.decode(ctx.decrypt(sk, y))).real[:10]
        want = resnet.forward_fp64(X, w)
        err = max(err, float(np.max(np.abs(got - want))))
        err_cheb = max(err_cheb, float(np.max(np.abs(got - resnet.forward_fp64(X, w, relu=cheb_relu)))))
        agree += int(np.argmax(got) == np.argmax(want))
    nkeys, kbytes = ctx.key_stats()
    n_boot = net.n_boot
    n_sparse = sum(1 for op in net.plan if op[0] == "boot" and op[2] is not net._boots.get((0, False)))
    del outs, gouts, cts, net, sk, pk
    release(ctx)
    return {"s_per_inference": secs / n_inputs, "eager_s_per_inference": eager_secs / n_inputs,
            "per_ciphertext_path_s_per_inference": plain_secs / n_inputs,
            "batched_s_per_inference": batch_secs / n_inputs, "batched_equals_one_by_one": batch_same,
            "eager_ms_by_step_kind": {k: round(v, 2) for k, v in sorted(kind_ms.items(), key=lambda kv: -kv[1])},
            "graph_equals_eager": same, "bootstrap_ms": boot_ms, "bootstrap_ms_by_kind": boot_ms_by,
            "bootstraps_per_inference": n_boot, "sparse_bootstraps_per_inference": n_sparse,
            "bootstrap_kernels": boot_kernels,
            "inputs": n_inputs, "prepare_and_keygen_s": round(t_prep, 2), "keys": nkeys, "key_bytes": kbytes,
            "max_abs_logit_vs_fp64_chebyshev_relu": err_cheb,
            "max_abs_logit_vs_fp64_exact_relu": err, "argmax_agrees": "%d/%d" % (agree, n_inputs),
            "levels": len(P["qbits"]), "paper_cpu_s_per_inference": 403}


def serving_timing(F, n_req=200, rate=4.0, max_active=12, frac_resnet=0.3):
    """The serving workload: Poisson arrivals (exponential gaps of mean 1/rate
    s from a seed), each request LeNet-5 (N = 2^15) or, with probability
    frac_resnet, ResNet-20 with bootstrapping (N = 2^16), both models on one
    continuous-batching server (fheon_server_*: each context on its own
    stream, their batches overlapping on the device, a layer step of one
    request alone replayed as a CUDA graph on pooled request buffers; the
    ResNet model is a program of layer, bootstrap, add and constant steps
    over three registers).
    Admission by memory: the budget holds the footprints of one ResNet-20 and
    three LeNet-5 requests (fheon_model_footprint), less than two ResNet-20
    footprints.  Requests are submitted when
    their arrival time has passed (host clock); latency = completion -
    arrival."""
    import torch
    from paper_2510_03996_gb300 import lenet, resnet
    kind = synth.rng(synth.SEED_BASE + 5, 802).random(n_req) < frac_resnet
    gaps = synth.rng(synth.SEED_BASE + 5, 801).exponential(1.0 / rate, n_req)
    arrive = np.cumsum(gaps) - gaps[0]
    # LeNet-5 on its context
    P = synth.params("lenet_n15")
    N = 1 << P["logN"]
    s1 = torch.cuda.Stream()
    c1 = F.Context(N, qbits=P["qbits"], pbits=P["pbits"], dnum=P["dnum"], scale=P["scale"], seed=P["seed"],
                   stream=s1.cuda_stream)
    w = lenet.weights(P["seed"])
    xs = [synth.image(P["seed"], 800 + i, (1, 28, 28)) for i in range(16)]
    sk, pk = c1.keygen()
    c1.relinkeygen(sk)
    ln = lenet.EncryptedLeNet(c1, w, lenet.relu_bounds(xs, w), c1.L, P["scale"])
    c1.rotkeygen(sk, ln.rotation_steps())
    m1 = c1.model(ln.layers)
    ct1 = [c1.encrypt(pk, c1.encode(lenet.pack_input(X, N // 2), c1.L, P["scale"]), nonce=i)
           for i, X in enumerate(xs)]
    c1.model_run(m1, ct1[0])  # warm-up
    # ResNet-20 on its context
    P = synth.params("resnet_n16")
    N = 1 << P["logN"]
    s2 = torch.cuda.Stream()
    c2 = F.Context(N, qbits=P["qbits"], pbits=P["pbits"], dnum=P["dnum"], scale=P["scale"], seed=P["seed"],
                   stream=s2.cuda_stream)
    w = resnet.weights(P["seed"])
    xs = [synth.image(P["seed"], 900 + i, (3, 32, 32), dist="normal") for i in range(4)]
    sk, pk = c2.keygen()
    rn = resnet.EncryptedResNet(c2, w, resnet.relu_bounds(xs, w), P["scale"])
    rn.keygen(sk)
    m2 = rn.model()
    ct2 = [c2.drop_level(c2.encrypt(pk, c2.encode(resnet.pack_input(X, N // 2), c2.L, P["scale"]), nonce=i),
                         rn.in_level) for i, X in enumerate(xs)]
    c2.model_run(m2, ct2[0])  # warm-up
    models = [(c1, m1, ct1), (c2, m2, ct2)]
    fp = [F.Context.model_footprint(m1, c1.ct_info(ct1[0])[0]), F.Context.model_footprint(m2, rn.in_level)]
    # the device memory left once both models' keys are resident (free, plus
    # what torch's cache holds unused), less a margin, bounded by one ResNet-20
    # and three LeNet-5 requests: below two ResNet-20 footprints, so that
    # ResNet-20 requests never take all of it and LeNet-5 requests keep flowing
    torch.cuda.synchronize()
    free_b, _ = torch.cuda.mem_get_info()
    avail = free_b + torch.cuda.memory_reserved() - torch.cuda.memory_allocated()
    budget = int(min(3 * fp[0] + fp[1], 0.8 * avail))
    srv = c1.server(max_active=max_active, mem_budget=budget)
    srv.set_graphs(True)  # single-request layer steps replay captured graphs on pooled buffers
    c1.sync()
    c2.sync()
    t0 = time.perf_counter()
    ids, done = {}, {}
    owner = {i: int(kind[i]) for i in range(n_req)}
    nxt = 0
    while len(done) < n_req:
        now = time.perf_counter() - t0
        while nxt < n_req and arrive[nxt] <= now:
            ctx, model, cts = models[owner[nxt]]
            ids[nxt] = srv.submit(model, cts[nxt % len(cts)])
            nxt += 1
        if len(ids) == len(done):
            time.sleep(max(0.0, min(0.01, arrive[nxt] - now)))
            continue
        if srv.step():
            now = time.perf_counter() - t0
            for k in list(ids):
                if k not in done and srv.result(ids[k]) is not None:
                    done[k] = now
    lat = np.array([done[k] - arrive[k] for k in range(n_req)])
    span = max(done.values()) - arrive[0]
    out = {"requests": n_req, "arrival_rate_per_s": rate,
           "models": "LeNet-5 (N=2^15) %d, ResNet-20 with bootstrapping (N=2^16) %d" % (n_req - kind.sum(), kind.sum()),
           "server": "one server over both contexts, their batches overlapping on two streams",
           "throughput_per_s": n_req / span, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
           "p99_ms": 1e3 * float(np.percentile(lat, 99)), "max_active": max_active,
           "mem_budget_bytes": budget, "device_bytes_available": avail,
           "footprint_bytes": {"lenet5": fp[0], "resnet20": fp[1]},
           "mem_waits": srv.model_stats(m1)["mem_waits"], "steps": srv.stats()["steps"],
           "graph_replayed_layer_steps": srv.graph_replays()}
    for which, name, m in ((0, "lenet5", m1), (1, "resnet20", m2)):
        sel = np.array([owner[k] == which for k in range(n_req)])
        if sel.any():
            out[name + "_p50_ms"] = 1e3 * float(np.percentile(lat[sel], 50))
            out[name + "_p99_ms"] = 1e3 * float(np.percentile(lat[sel], 99))
        out[name + "_max_batch"] = srv.model_stats(m)["max_batch"]
    srv.close()
    del models, ct1, ct2, ln, rn, m1, m2
    release(c1, c2)
    return out


def conv_layer_timing(F, iters=200):
    """Packed special conv of the 1x28x28, 5x5, pad 2 layer at N = 2^13 (24 tap
    rotations + 25 plaintext products + one rescale), eager and as a replayed
    CUDA graph, in microseconds per layer."""
    import torch
    P = synth.params("conv_n13")
    N = 1 << P["logN"]
    s = torch.cuda.Stream()
    ctx = F.Context(N, qbits=P["qbits"], pbits=P["pbits"], dnum=P["dnum"], scale=P["scale"], seed=P["seed"],
                    stream=s.cuda_stream)
    H = W = 28
    k = 5
    sk, pk = ctx.keygen()
    ctx.rotkeygen(sk, ctx.conv2d_rotation_steps(1, 1, k, 1, (k - 1) // 2, H, W))
    x = np.zeros(N // 2)
    x[:H * W] = synth.image(P["seed"], 0, (1, H, W)).reshape(-1)
    ct = ctx.encrypt(pk, ctx.encode(x, ctx.L, P["scale"]), nonce=1)
    layer = ctx.conv2d_prepare(1, k, 1, 2, H, W, synth.conv_kernel(P["seed"], 1, (1, k, k)), [0.0], ctx.L, P["scale"])
    out = ctx.ct_create(ctx.L)
    res = {}
    for name, fn in (("eager", ctx.conv2d_apply), ("graph", ctx.conv2d_apply_graph)):
        for _ in range(3):
            fn(layer, ct, out)
        ctx.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("conv_" + name)
        e0.record(s)
        for _ in range(iters):
            fn(layer, ct, out)
        e1.record(s)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        res[name + "_us_per_layer"] = 1e3 * e0.elapsed_time(e1) / iters
    ctx.sync()
    layer.close()
    del out, ct, sk, pk
    release(ctx)
    return res


def run_gpu(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2510_03996_gb300 import fheon as F

    F.use_torch_allocator()
    P = synth.params(WORKLOAD)
    N = 1 << P["logN"]
    stream = torch.cuda.current_stream()
    ctx = F.Context(N, qbits=P["qbits"], pbits=P["pbits"], dnum=P["dnum"], scale=P["scale"], seed=P["seed"],
                    stream=stream.cuda_stream)
    levels, steps = synth.rotation_workload(P["seed"], n_ct=args.n_ct)
    sk, pk = ctx.keygen()
    t0 = time.time()
    ctx.rotkeygen(sk, sorted(set(steps)))
    ctx.sync()
    nkeys, kbytes = ctx.key_stats()
    t_keys = time.time() - t0
    z = synth.uniform_slots(P["seed"], 3, N // 2)
    pt = ctx.encode(z, ctx.L, P["scale"])
    ins, outs = [], []
    for i, lv in enumerate(levels):
        ct = ctx.encrypt(pk, pt, nonce=i)
        ins.append(ctx.drop_level(ct, lv))
        outs.append(ctx.ct_create(lv, P["scale"]))
        del ct
    ctx.sync()

    def step():
        ctx.rotate_batch(ins, outs, steps)

    # integer peaks of this GPU: the rate of each modular step the ALU-bound
    # kernels are built from (fheon_alu_peak), the denominators of their rooflines
    alu_rates = {k: ctx.alu_peak(k) for k in F.Context.PEAK_KINDS}

    if args.schedule < 0:
        # the library's autotuner picks the key-switching schedule for this batch
        schedule, tune_ms = ctx.autotune_schedule(ins, outs, steps, reps=2)
    else:
        ctx.set_schedule(args.schedule)
        schedule, tune_ms = args.schedule, {}

    for _ in range(args.warmup):
        step()
    ctx.sync()
    if world > 1:
        torch.distributed.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    ms_total = ev0.elapsed_time(ev1)
    # per-kernel times: the same steps once more, with a CUDA event recorded
    # after every launch on the launching stream (the headline above runs
    # without that instrumentation)
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ctx.profile_begin()
    ev2.record(stream)
    for _ in range(args.steps):
        step()
    ev3.record(stream)
    prof = ctx.profile_end()
    torch.cuda.synchronize()
    ms_profiled = ev2.elapsed_time(ev3)
    value = replica_rate(len(levels) * args.steps, ms_total / 1e3, world)
    ms_total = barrier_max(ms_total, world)
    ms_step = ms_total / args.steps

    # e2e: every step uploads its inputs from pinned host memory, rotates them and
    # downloads the results, through the library's calls.  The batch's
    # ciphertexts sit back to back in one device allocation
    # (fheon_ct_create_batch), so a step is one host-to-device and one
    # device-to-host copy; the copies run on two copy streams and overlap the
    # key switching of the neighbouring steps (two device batches, ordered by
    # events).
    words = sum(2 * lv * N for lv in levels)
    host_in = torch.empty(words, dtype=torch.int64, pin_memory=True)
    host_out = torch.empty(words, dtype=torch.int64, pin_memory=True)
    depth = args.e2e_depth
    bufs = [(ctx.ct_create_batch(levels, P["scale"]), ctx.ct_create_batch(levels, P["scale"])) for _ in range(depth)]
    for c, b in zip(ins, bufs[0][0]):
        ctx.drop_level(c, ctx.ct_info(c)[0], out=b)
    ctx.ct_download_many_async(bufs[0][0], host_in.data_ptr())
    ctx.sync()
    h2d = d2h = words * 8
    s_up, s_dn = torch.cuda.Stream(), torch.cuda.Stream()

    def e2e_run(nsteps):
        ev_comp, ev_dn = {}, {}
        for k in range(nsteps):
            bi, bo = bufs[k % depth]
            if k >= depth:
                s_up.wait_event(ev_comp[k - depth])  # the inputs of step k-depth are consumed
            ctx.ct_upload_many_async(bi, host_in.data_ptr(), s_up.cuda_stream)
            up = torch.cuda.Event()
            up.record(s_up)
            stream.wait_event(up)
            if k >= depth:
                stream.wait_event(ev_dn[k - depth])  # the outputs of step k-depth are read out
            ctx.rotate_batch(bi, bo, steps)
            ev_comp[k] = torch.cuda.Event(enable_timing=True)
            ev_comp[k].record(stream)
            s_dn.wait_event(ev_comp[k])
            ctx.ct_download_many_async(bo, host_out.data_ptr(), s_dn.cuda_stream)
            ev_dn[k] = torch.cuda.Event()
            ev_dn[k].record(s_dn)
        torch.cuda.synchronize()
        # the key switching of each step ends this long after the previous one's
        return [ev_comp[k - 1].elapsed_time(ev_comp[k]) for k in range(1, nsteps)]

    e2e_steps = max(4, 2 * args.steps)
    e2e_run(depth)  # warm-up: every device batch once (its rotation plan is made then)
    with ClockSampler(local_rank) as e2e_clk:
        t0 = time.perf_counter()
        e2e_ms = e2e_run(e2e_steps)
        e2e_secs = time.perf_counter() - t0
    e2e_value = replica_rate(len(levels) * e2e_steps, e2e_secs, world)
    # the pipelined downloads are the batch's results
    first = host_out[:2 * levels[0] * N].numpy().view(np.uint64).reshape(2, levels[0], N)
    e2e_ok = bool(np.array_equal(first, ctx.ct_download(outs[0])))

    # roofline of the dominant kernel, from the live per-launch events
    pk_, src = peaks()
    launches = sum(v[0] for v in prof.values())
    mods = ctx.moduli
    costs = [algorithmic_costs(N, ctx.L, ctx.K, ctx.alpha, lv, q_lazy=max(mods[:ctx.L]) < (1 << 54),
                               p_lazy=max(mods[ctx.L:]) < (1 << 54)) for lv in levels]
    roofs = rooflines(prof, costs, args.steps, float(pk_["hbm_gbs"]), alu_rates)
    dom_name = max(prof.items(), key=lambda kv: kv[1][1])[0]
    roof = dict(roofs[dom_name])
    traffic = None
    if TRAFFIC_OVER_MIN.get(dom_name):
        mb = sum(c["kernels"][dom_name].get("min_bytes", 0) for c in costs)
        traffic = TRAFFIC_OVER_MIN[dom_name] * mb / (prof[dom_name][0] / args.steps)
    roof.update({"kernel": dom_name, "traffic": traffic,
                 "traffic_source": "ncu DRAM bytes of the 16-ciphertext case over the kernel's minimum bytes, "
                                   "times this workload's minimum bytes per launch" if traffic else None,
                 "peak_source": ("%s copy bandwidth" % src) if roof["bound"] == "hbm" else
                 "measured in this run (fheon_alu_peak): the kernel's mix of butterflies and conversion "
                 "multiply-accumulates at their measured rates",
                 "kernel_times": "CUDA events after every launch, in a pass of the same %d steps right after "
                                 "the timed region (%.2f ms per step there)" % (args.steps, ms_profiled / args.steps)})
    kernels = {k: {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / sum(x[1] for x in prof.values()), 4),
                   "frac": round(roofs.get(k, {}).get("frac", 0.0), 4), "bound": roofs.get(k, {}).get("bound")}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}

    comparisons = None
    # single-GPU diagnostics beside the timed step: each replica would only repeat them
    if not args.no_comparisons and world == 1:
        per_ct = per_ciphertext_rate(ctx, ins, outs, steps, stream)
        # the rotation workload's keys and batches are done with: hand their memory
        # back before the other workloads build their own contexts
        del ins, outs, bufs, host_in, host_out
        release(ctx)
        comparisons = {"per_ciphertext_path": per_ct,
                       "conv_n13_layer": conv_layer_timing(F),
                       "lenet5_n15": lenet_timing(F),
                       "resnet20_n16": resnet_timing(F),
                       "serving_mixed": serving_timing(F, n_req=args.serve_requests)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate1, done1, secs1, used = OracleRunner(P, steps[0]).rate(levels, budget_s=args.cpu_budget)
        rate, done, secs, cores = oracle_all_cores(P, steps[0], levels)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d rotations of the workload's first items at once, one process per host core, "
                         "slowest %.1f s; on one core: %d rotations (levels %s) in %.1f s" %
                         (done, secs, done1, used, secs1),
               "single_core_value": rate1}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": "batched rotation, N=2^16, 24x50-bit Q + 4x60-bit P, dnum 6, %d ciphertexts "
                                       "at levels U{4..24}, steps U[1,2^15), one key per step" % len(levels),
                           "keys": nkeys, "key_bytes": kbytes, "keygen_s": round(t_keys, 2),
                           "ks_schedule": schedule,
                           "autotune_ms_per_batch": {str(k): round(v, 3) for k, v in tune_ms.items()},
                           "mean_level": float(np.mean(levels)), "parallelism": "replicas" if world > 1 else "none",
                           "l2": "inputs larger than L2 (keys %.1f GB)" % (kbytes / 1e9)},
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "steps": e2e_steps, "pipelined": "one upload and one download per step (contiguous ciphertext "
                                                          "batch) on two copy streams, overlapping the key switching of "
                                                          "neighbouring steps; %d device batches in flight" % depth,
                        "result_matches": e2e_ok,
                        "steps_ms": step_summary(e2e_ms), "clocks": e2e_clk.summary()},
                "clocks": clk.summary(), "gpu_launches": launches, "kernels": kernels,
                "alu_peaks_tmodmul_s": {k: round(v / 1e12, 4) for k, v in alu_rates.items()},
                "comparisons": comparisons}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fheon", choices=["fheon", "reference"])
    ap.add_argument("--n-ct", type=int, default=256)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparisons", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--e2e-depth", type=int, default=4,
                    help="device batches of the end-to-end pipeline (uploads run up to depth-1 steps ahead)")
    ap.add_argument("--schedule", type=int, default=-1,
                    help="key-switching schedule bits (default: the library's autotuner picks)")
    args = ap.parse_args()
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
