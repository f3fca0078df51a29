"""Benchmark: encrypted MNIST-shaped CNN inferences/s on one GB300 (and N replicas under torchrun).

Workload (the paper's evaluation network, §5 / Table 2, with the chain N=8192, primes
[31,26,26,26,26,26,26,31], scale 2^26): 28x28 seeded uniform image, im2col-encoded and encrypted;
conv 4x7x7 stride 3 -> square -> FC 256->64 -> square -> FC 64->10 on seeded N(0, 0.1) weights.
A step is one batch of B encrypted inferences (B requests, default 256) through the whole hot path
(conv rotations, pack, relinearized squares, two hoisted vector x matrix products) in the batched
schedule, where every stage runs once for the whole batch; inputs are resident in HBM. Per step the
kernels stream the Galois keys plus several GB of per-request key-switch scratch (~2 GB at B = 64),
far more than the 129 MB L2, so no L2 flush is added. The plain path (one request per step) is timed alongside.
`e2e` times the batched step through the C ABI on serialized ciphertexts (tcks_cnn_forward_wire), the
exchange of the serving scenario: one copy of the B clients' seeded inputs (c0 bit-packed + the seed of
c1) from pinned host memory, unpacking and c1 regenerated on the device, the batched schedule, the
outputs packed on the device and copied back, all inside the timed region. `e2e_limbs` is the same
with 64-bit limbs in and out (tcks_cnn_forward_host).

--impl reference times the CPU oracle (the plain CKKS written from the definitions) on the host
cores, one inference per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile

# Load every kernel of the process when CUDA starts instead of on its first launch: a kernel first used
# in the middle of the serving trace (a shape the warm-up did not reach) would load there and stall
# every lane for tens of milliseconds (measured: served p99 190 ms with on-demand loading, 31 ms here).
os.environ.setdefault("CUDA_MODULE_LOADING", "EAGER")
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encrypted-CNN inferences/s + p99 latency (served vs plain); NTT/keyswitch GB/s"
LOG_N, BITS, SCALE = 13, [31, 26, 26, 26, 26, 26, 26, 31], 2.0 ** 26
SEED_IMG, SEED_W, SEED_ENC = 3, 4, 77
WORKLOAD = ("encrypted MNIST-shaped CNN (conv 4x7x7/3 -> sq -> FC256->64 -> sq -> FC64->10), CKKS N=8192, "
            "primes [31,26x6|31], scale 2^26, Galois keys trimmed to their levels")


# ----------------------------------------------------------------------------- distributed --
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, local):
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if dist.is_nccl_available() else "gloo"
        dist.init_process_group(backend=backend)
    return torch


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(world, x: float) -> float:
    """The largest x over the ranks (the slowest rank's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, batch: int, steps: int, total_ms: float) -> float:
    """Whole-job inferences/s: every rank runs `steps` batches of `batch` independent requests (replicas,
    no exchange), over the slowest rank's time (total_ms, already the max over ranks)."""
    return world * batch * steps / (total_ms / 1e3)


# ------------------------------------------------------------------------------------ clocks --
class Clocks:
    """nvidia-smi samples (every 50 ms) during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 10:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        load = [r for r in rows if (num(r[4]) or 0) >= 50] or rows
        sm = [num(r[1]) for r in load if num(r[1]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[6:10]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": num(rows[0][2]), "reasons": sorted(reasons),
                "samples": len(rows), "samples_under_load": len(load),
                "power_w_max": max((num(r[3]) or 0) for r in rows)}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def ncu_traffic(kernel: str, config: dict):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary (profiles/ncu_traffic.json),
    if it was taken on the current sources of the files that define and launch the kernel and on the
    same bench configuration; None otherwise."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    ent = d.get("kernels", {}).get(kernel)
    if not ent or ent.get("src_sha") != source_digest(ent.get("files", [])):
        return None
    if any(config.get(k) != v for k, v in ent.get("config", {}).items()):
        return None
    return ent.get("dram_bytes_per_launch")


def source_digest(files) -> str:
    """sha256 (16 hex digits) over the named files of the library's csrc directory, in order."""
    import hashlib
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_2104_03152_gb300", "csrc")
    for f in files:
        h.update(f.encode())
        h.update(open(os.path.join(src, f), "rb").read())
    return h.hexdigest()[:16]


# ---------------------------------------------------------------------------------- GPU arm --
def gpu_setup(torch, batch, double_hoist, rect=False, conv_hoist=False, conv_shared=False, conv_pack=False,
              merged=False, fold=False):
    import paper_2104_03152_gb300 as tk
    from paper_2104_03152_gb300 import inputs

    tk.lib(build_if_missing=True)
    stream = torch.cuda.Stream()
    flags = (tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE | (tk.TCKS_DOUBLE_HOIST if double_hoist else 0)
             | (tk.TCKS_RECT_DIAG if rect else 0) | (tk.TCKS_CONV_HOIST if conv_hoist else 0)
             | (tk.TCKS_CONV_SHARED if conv_hoist and conv_shared else 0)
             | (tk.TCKS_CONV_PACK if conv_hoist and conv_pack else 0)
             | (tk.TCKS_CONV_FOLD if conv_hoist and conv_shared and conv_pack and fold else 0)
             | (tk.TCKS_MERGED_RESCALE if merged else 0))
    ctx = tk.Context(tk.Params(LOG_N, BITS, SCALE), seed=inputs.SEED_KEYS, flags=flags, stream=stream.cuda_stream)
    w = inputs.cnn_weights(SEED_W)
    model = tk.CNN(ctx, w["conv_w"], w["conv_b"], w["fc1_w"], w["fc1_b"], w["fc2_w"], w["fc2_b"], windows=64)
    model.gen_keys()
    imgs = [inputs.mnist_like_image(SEED_IMG + i) for i in range(batch)]
    cts = []
    for i, img in enumerate(imgs):
        v, _ = tk.im2col_encode(img, 7, 7, 3, ctx.slots)
        cts.append(ctx.encrypt_values(v, SEED_ENC + i))
    ctx.synchronize()
    return tk, ctx, model, cts, stream, imgs, w


def timed(torch, stream, fn, steps):
    """CUDA-event times (ms) of `steps` calls of fn on `stream`, one event pair per step."""
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    with torch.cuda.stream(stream):
        evs[0].record(stream)
        for k in range(steps):
            fn()
            evs[k + 1].record(stream)
    stream.synchronize()
    return [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)], evs[0].elapsed_time(evs[-1])


def run_gpu(args, world, rank, local):
    torch = dist_init(world, local)
    B = args.batch
    rect = args.fc_form == "rect"
    tk, ctx, model, cts, stream, imgs, w = gpu_setup(torch, B, args.double_hoist, rect, bool(args.conv_hoist),
                                                     bool(args.conv_shared), bool(args.conv_pack),
                                                     bool(args.merged_rescale), bool(args.conv_fold))
    # correctness guard: the decrypted logits of every request must match the FP64 network, and the
    # batched outputs must equal the single-request path bit for bit
    outs = model.forward_batch(cts)
    max_err = 0.0
    for i in (0, B - 1):
        logits = ctx.decrypt_values(outs[i], 10)
        max_err = max(max_err, float(np.max(np.abs(logits - plain_cnn(imgs[i], w)))))
        assert np.array_equal(outs[i].export(), model.forward(cts[i]).export()), "batched != single"
    # the timed step: the whole batch on one contiguous device buffer (inputs resident in HBM)
    L_in, N_ = cts[0].level, ctx.N
    d_in = torch.empty((B, 2, L_in, N_), dtype=torch.int64, device="cuda")
    for i, c in enumerate(cts):
        d_in[i].copy_(torch.from_numpy(c.export().view(np.int64)))
    d_out = torch.empty((B, 2, outs[0].level, N_), dtype=torch.int64, device="cuda")
    d_in_ptr, d_out_ptr = d_in.data_ptr(), d_out.data_ptr()
    torch.cuda.synchronize()
    model.forward_device(d_in_ptr, B, d_out_ptr)
    ctx.synchronize()
    for i in (0, B - 1):
        assert np.array_equal(d_out[i].cpu().numpy().view(np.uint64), outs[i].export()), "device batch != batched"
    for _ in range(args.warmup):
        model.forward_device(d_in_ptr, B, d_out_ptr)
    ctx.synchronize()
    # launch shape: the hand-tuned default, then the autotuner's choice (kept for the timed region)
    _, hand_ms = timed(torch, stream, lambda: model.forward_device(d_in_ptr, B, d_out_ptr), 3)
    tune_cache = os.path.join(tempfile.gettempdir(), "tcks_autotune.json")
    tuned = model.autotune(B, tune_cache if args.tune_cache else None)
    for _ in range(2):
        model.forward_device(d_in_ptr, B, d_out_ptr)
    _, tuned_ms = timed(torch, stream, lambda: model.forward_device(d_in_ptr, B, d_out_ptr), 3)
    tune = {"limb_threads": tuned[0],
            "accumulation_requests_per_thread": tuned[1] if tuned[1] else
            "default: 4 where a plan's keys sit at its level 4 or 5, else 2",
            "accumulation_form": "per-thread loads" if tuned[2] == 0 else
            "operands staged in shared memory by bulk copies, %d elements per CTA x %d stages"
            % {1: (256, 2), 2: (256, 3), 3: (128, 3), 4: (128, 4)}[tuned[2]],
            "hand_tuned_ms_per_step": hand_ms / 3, "autotuned_ms_per_step": tuned_ms / 3,
            "searched": "limb-kernel CTA size {N/64, N/32, N/16 per slice} x accumulation requests per thread "
                        "{default, 2, 4, 1} x accumulation form {per-thread loads, staged by bulk copies: 256 x 2, "
                        "256 x 3, 128 x 3, 128 x 4 elements per CTA x stages}"}
    ctx.synchronize()
    # plain path: one request per step
    plain_steps = max(3, min(args.steps, 10))
    for _ in range(2):
        model.forward(cts[0])
    plain_times, plain_total = timed(torch, stream, lambda: model.forward(cts[0]), plain_steps)
    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    n0 = tk.launch_count()
    tk.profile_start()
    torch.cuda.nvtx.range_push("timed")
    per_step, total_ms = timed(torch, stream, lambda: model.forward_device(d_in_ptr, B, d_out_ptr), args.steps)
    torch.cuda.nvtx.range_pop()
    tk.profile_stop()
    dh_records = tk.profile_records("vecmat_dh_acc")
    launches = tk.launch_count() - n0
    barrier(world)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = reduce_max(world, total_ms)
    prof = tk.profile_read(with_ops=True)
    # e2e through the C ABI with pinned host buffers: B inputs in, batched forward, B outputs out
    L, N = cts[0].level, ctx.N
    host_in = torch.empty(B * 2 * L * N, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    host_in = host_in.reshape(B, 2, L, N)
    for i, c in enumerate(cts):
        host_in[i] = c.export()
    out_words = 2 * outs[0].level * N
    host_out = torch.empty(B * out_words, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    host_out = host_out.reshape(B, out_words)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(3, args.steps // 2)
    out_view = host_out.reshape(B, 2, outs[0].level, N)
    for _ in range(e2e_steps):
        model.forward_host(host_in, out_view)
    torch.cuda.synchronize()
    e2e_s = reduce_max(world, time.perf_counter() - t0)
    # e2e on the wire (the client-server exchange of the serving scenario): the clients' secret-key
    # ciphertexts in their seeded serialized form (c0 bit-packed + the seed of c1) in, the serialized
    # outputs out, through tcks_cnn_forward_wire
    full_sz, seeded_sz, out_sz = model.wire_sizes()
    wire_in = torch.empty(B * seeded_sz, dtype=torch.uint8, pin_memory=True).numpy()
    wire_out = torch.empty(B * out_sz, dtype=torch.uint8, pin_memory=True).numpy()
    for i, img in enumerate(imgs):
        v, _ = tk.im2col_encode(img, 7, 7, 3, ctx.slots)
        ct_s = ctx.encrypt_symmetric(ctx.encode(v), SEED_ENC + 5000 + i, SEED_ENC + 9000 + i)
        wire_in[i * seeded_sz:(i + 1) * seeded_sz] = np.frombuffer(ct_s.serialize_seeded(SEED_ENC + 5000 + i),
                                                                     dtype=np.uint8)
    model.forward_wire(wire_in, B, wire_out)
    for i in (0, B - 1):
        back = ctx.ct_deserialize(wire_out[i * out_sz:(i + 1) * out_sz].tobytes())
        err = float(np.max(np.abs(ctx.decrypt_values(back, 10) - plain_cnn(imgs[i], w))))
        assert err < 1e-2, f"wire output {i} off by {err}"
        max_err = max(max_err, err)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        model.forward_wire(wire_in, B, wire_out)
    torch.cuda.synchronize()
    wire_sync_s = reduce_max(world, time.perf_counter() - t0)
    # the same exchange pipelined (tcks_cnn_pipe_*): batch k's input copy overlaps batch k-1's network;
    # every batch still copies its serialized inputs in and its serialized outputs out
    pipe = model.pipe(B, seeded_sz)
    wire_outs = [wire_out, torch.empty(B * out_sz, dtype=torch.uint8, pin_memory=True).numpy()]
    pipe.wait(pipe.submit(wire_in, wire_outs[1]))
    assert np.array_equal(wire_outs[1], wire_out), "pipelined output != forward_wire output"
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tickets = []
    for k in range(e2e_steps):
        tickets.append(pipe.submit(wire_in, wire_outs[k % 2]))
        if k >= 1:
            pipe.wait(tickets[k - 1])
    pipe.wait(tickets[-1])
    torch.cuda.synchronize()
    wire_s = reduce_max(world, time.perf_counter() - t0)
    del pipe
    # the same batched step with one ModDown per rotation (the schedule bit-identical to rotating
    # each diagonal's ciphertext separately), for comparison
    single = {}
    base = tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE
    dh_flag = tk.TCKS_DOUBLE_HOIST if args.double_hoist else 0

    def time_model(mdl, label):
        mdl.forward_device(d_in_ptr, B, d_out_ptr)
        _, tot = timed(torch, stream, lambda: mdl.forward_device(d_in_ptr, B, d_out_ptr), 3)
        single[label] = {"value": B * 3 / (tot / 1e3), "unit": "inferences/s", "ms_per_step": tot / 3}
    form = "rectangular" if rect else "square"
    conv = CONV_LABEL[conv_form(args)]
    run_flags = ctx.flags
    if args.merged_rescale:  # the same network with the ModDown and the rescale as two roundings
        ctx.set_flags(run_flags & ~tk.TCKS_MERGED_RESCALE)
        time_model(model, f"{form} FC layers, {conv}, ModDown and rescale as two roundings")
        ctx.set_flags(run_flags)
    if args.double_hoist:
        ctx.set_flags(base)
        time_model(model, f"{form} FC layers, {conv}, one ModDown per FC rotation")
        ctx.set_flags(run_flags)

    def other(flags, label):  # another network layout on the same context
        ctx.set_flags(base | dh_flag | flags)
        alt = tk.CNN(ctx, w["conv_w"], w["conv_b"], w["fc1_w"], w["fc1_b"], w["fc2_w"], w["fc2_b"], windows=64)
        ctx.set_flags(base | dh_flag)
        alt.gen_keys()
        time_model(alt, label)
    if conv_form(args) == "shared+pack+fold":
        other((tk.TCKS_RECT_DIAG if rect else 0) | tk.TCKS_CONV_SHARED | tk.TCKS_CONV_PACK,
              f"{form} FC layers, {CONV_LABEL['shared+pack']}")
    if conv_form(args).startswith("shared+pack"):
        other((tk.TCKS_RECT_DIAG if rect else 0) | tk.TCKS_CONV_SHARED, f"{form} FC layers, {CONV_LABEL['shared']}")
    if conv_form(args).startswith("shared"):
        other((tk.TCKS_RECT_DIAG if rect else 0) | tk.TCKS_CONV_HOIST, f"{form} FC layers, {CONV_LABEL['hoist']}")
    if args.conv_hoist:
        other(tk.TCKS_RECT_DIAG if rect else 0, f"{form} FC layers, rotate-and-add convolution chain")
    if rect:
        other(0, "square FC layers, rotate-and-add convolution chain")
    c4 = run_c4(torch, tk, args) if args.c4 else None
    serving = None
    if args.serve_seconds > 0:
        mix = args.serve_mix if c4 else 0.0
        clients = serving_clients(torch, tk, args, (ctx, model, cts), (c4["ctx"], c4["mat"], c4["cts"]) if c4 else None)
        pct = lambda a, p: float(np.percentile(a, p) * 1e3) if len(a) else None

        def summary(lat, kind, thr):
            d = {"throughput": thr, "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "requests": len(lat)}
            for k in ("cnn", "vm"):
                sel = lat[kind == k]
                if len(sel):
                    d[k] = {"requests": len(sel), "p50_ms": pct(sel, 50), "p99_ms": pct(sel, 99)}
            return d
        traces = []
        total_s = args.serve_warmup + args.serve_seconds
        for rate in [float(x) for x in args.serve_rate.split(",")]:
            arr = poisson_arrivals(rate, total_s, 8)
            rng = np.random.default_rng(9)
            kinds = np.where(rng.uniform(size=len(arr)) < mix, "vm", "cnn")
            who = np.array([rng.integers(len(clients[k])) for k in kinds])
            lat_s, kind_s, thr_s, st = serve_trace(tk, clients, arr, kinds, who, args.serve_batch, args.serve_warmup)
            n_p = len(arr) if args.plain_requests <= 0 else min(len(arr), args.plain_requests)
            lat_p, kind_p, thr_p = plain_trace(tk, clients, arr[:n_p], kinds[:n_p], who[:n_p], args.serve_warmup)
            traces.append({"offered_rate": rate, "seconds": args.serve_seconds, "warmup_seconds": args.serve_warmup,
                           "requests": int(np.sum(arr >= args.serve_warmup)),
                           "served": dict(summary(lat_s, kind_s, thr_s), max_batch_per_stage=args.serve_batch,
                                          max_in_flight=1024, hbm_budget_gb=200,
                                          hbm_resident_gb=st["bytes_resident"] / 1e9),
                           "plain": dict(summary(lat_p, kind_p, thr_p),
                                         trace_requests=int(np.sum(arr[:n_p] >= args.serve_warmup)))})
        serving = {"mix": {"cnn": 1.0 - mix, "vm": mix}, "vm_workload": C4_WORKLOAD if c4 else None,
                   "clients": {"cnn": len(clients["cnn"]), "vm": len(clients["vm"]),
                               "key_sets": "one context (own secret, relinearization and Galois keys) per client"},
                   "latency": "arrival -> result exported to the host", "traces": traces}
        del clients
    if c4:
        for k in ("ctx", "mat", "cts"):
            c4.pop(k)
    word = 32 if max(ctx.primes) < 2 ** 31 else 64
    bfly_peak = tk.calibrate_butterflies(word)
    mac_peak = tk.calibrate_macs(word)
    dh_peaks = {ell: tk.calibrate_dh_macs(ell) for ell in sorted({t & 0xFF for t, _, _ in dh_records})}
    primitives = primitives_summary(torch, tk) if args.primitives else None
    return dict(galois_keys=len(model.galois_steps()), single=single, c4=c4, primitives=primitives, bfly_peak=bfly_peak,
                mac_peak=mac_peak, dh_records=dh_records, dh_peaks=dh_peaks, word=word, tune=tune, serving=serving, total_ms=total_ms, per_step=per_step, prof=prof, launches=launches, clocks=clk, e2e_s=e2e_s,
                e2e_steps=e2e_steps, h2d=host_in.nbytes, d2h=host_out.nbytes, max_err=max_err, wire_s=wire_s,
                wire_sync_s=wire_sync_s,
                wire_h2d=wire_in.nbytes + 8 * B, wire_d2h=wire_out.nbytes + 4, wire_sizes=(seeded_sz, out_sz),
                plain_ms=plain_total / plain_steps, plain_times=plain_times)


def poisson_arrivals(rate: float, seconds: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            return np.array(out)
        out.append(t)


def _finish(tk, ctx, ct, hosts):
    """Export a result to the host (the end of a request's latency)."""
    key = (ctx.N, ct.info()[0])
    if key not in hosts:
        hosts[key] = np.zeros((2, key[1], ctx.N), dtype=np.uint64)
    h = hosts[key]
    tk.check(tk.lib().tcks_ct_export(ct.h, tk._p(h), h.size))


def serving_clients(torch, tk, args, cnn0, vm0):
    """The client population of the serving trace: args.cnn_clients CNN clients and args.vm_clients
    vector x matrix clients, each with its own key set (its own context, key seed SEED_KEYS + client),
    model or matrix, and a pool of its own encrypted inputs. cnn0 / vm0 are client 0 of each kind."""
    from paper_2104_03152_gb300 import inputs
    out = {"cnn": [cnn0], "vm": [vm0] if vm0 else []}
    w = inputs.cnn_weights(SEED_W)
    ctx0 = cnn0[0]
    for c in range(1, args.cnn_clients):
        st = torch.cuda.Stream()
        ctx = tk.Context(tk.Params(LOG_N, BITS, SCALE), seed=inputs.SEED_KEYS + c, flags=ctx0.flags,
                         stream=st.cuda_stream)
        ctx._torch_stream = st
        model = tk.CNN(ctx, w["conv_w"], w["conv_b"], w["fc1_w"], w["fc1_b"], w["fc2_w"], w["fc2_b"], windows=64)
        model.gen_keys()
        pool = []
        for i in range(4):
            v, _ = tk.im2col_encode(inputs.mnist_like_image(SEED_IMG + 100 * c + i), 7, 7, 3, ctx.slots)
            pool.append(ctx.encrypt_values(v, SEED_ENC + 100 * c + i))
        out["cnn"].append((ctx, model, pool))
    if vm0:
        vctx0 = vm0[0]
        for c in range(1, args.vm_clients):
            st = torch.cuda.Stream()
            ctx = tk.Context(tk.Params(14, [60, 40, 40, 60], 2.0 ** 40), seed=inputs.SEED_KEYS + 1000 + c,
                             flags=vctx0.flags, stream=st.cuda_stream)
            ctx._torch_stream = st
            ctx.gen_galois_keys([ctx.slots - C4_ROWS] + list(range(1, C4_COLS)) + [C4_COLS << j for j in range(4)])
            mat = ctx.matrix_encode_rect(inputs.random_matrix(C4_ROWS, C4_COLS, 7, 0.05), level=3)
            pool = []
            for i in range(4):
                z = np.zeros(ctx.slots)
                z[:C4_ROWS] = inputs.normal_slots(C4_ROWS, 6 + 1000 * (100 * c + i))
                pool.append(ctx.encrypt_values(z, 600 + 100 * c + i))
            out["vm"].append((ctx, mat, pool))
    torch.cuda.synchronize()
    return out


def serve_trace(tk, clients, arrivals, kinds, who, max_batch, warmup_s):
    """Continuous batching over one lane per client (a CNN or a vector x matrix product on the client's
    own key set), all under one HBM budget: requests are submitted when their arrival time passes and
    join their lane at its next launch; latency = arrival -> result exported to the host. Requests
    arriving in the first warmup_s seconds are served but not counted."""
    srv = tk.Server(hbm_budget_bytes=200 << 30, max_in_flight=1024, max_batch=max_batch)
    lane_of = {}
    for kind, lst in clients.items():
        for c, (ctx, model, pool) in enumerate(lst):
            lane_of[(kind, c)] = srv.add_cnn(model) if kind == "cnn" else srv.add_vecmat(model)
    hosts, pending, lat, lat_kind = {}, {}, [], []
    i, total, finished = 0, len(arrivals), 0
    t0 = time.perf_counter()
    while finished < total:
        now = time.perf_counter() - t0
        while i < total and arrivals[i] <= now:
            k, c = kinds[i], who[i]
            pool = clients[k][c][2]
            pending[srv.submit(lane_of[(k, c)], pool[i % len(pool)])] = (arrivals[i], k, c)
            i += 1
        st = srv.stats()
        if st["queued"] + st["in_flight"] == 0:
            time.sleep(max(0.0, min(arrivals[i] - now, 0.01)) if i < total else 0.0)
            continue
        srv.step()
        for rid in srv.poll():
            a, k, c = pending.pop(rid)
            _finish(tk, clients[k][c][0], srv.take(rid, clients[k][c][0]), hosts)
            finished += 1
            if a >= warmup_s:
                lat.append(time.perf_counter() - t0 - a)
                lat_kind.append(k)
    span = time.perf_counter() - t0 - warmup_s
    stats = srv.stats()
    return np.array(lat), np.array(lat_kind), len(lat) / span, stats


def plain_trace(tk, clients, arrivals, kinds, who, warmup_s):
    """The plain path on the same trace: one request at a time in arrival order, each on its client's
    key set; latencies counted after the warm-up as in serve_trace."""
    hosts, lat, lat_kind = {}, [], []
    t0 = time.perf_counter()
    for i, a in enumerate(arrivals):
        now = time.perf_counter() - t0
        if now < a:
            time.sleep(a - now)
        k, c = kinds[i], who[i]
        ctx, model, pool = clients[k][c]
        x = pool[i % len(pool)]
        out = model.forward(x) if k == "cnn" else x.vecmat_plain(model)
        _finish(tk, ctx, out, hosts)
        if a >= warmup_s:
            lat.append(time.perf_counter() - t0 - a)
            lat_kind.append(k)
    span = time.perf_counter() - t0 - warmup_s
    return np.array(lat), np.array(lat_kind), len(lat) / span if span > 0 else 0.0


# ------------------------------------------------------ vector x plain matrix at full size --
C4_ROWS, C4_COLS = 4096, 256
C4_WORKLOAD = ("encrypted 4096-dim N(0,1) vector x plain 4096x256 N(0,0.05) matrix (diagonal method, hoisted "
               "rotations, input replicated by one rotation), CKKS N=16384, primes [60,40,40|60], scale 2^40")


def run_c4(torch, tk, args):
    """The 4096x256 product for a batch of 64 vectors: the form given by --c4-form (rectangular
    diagonals: 255 hoisted rotations + 4 rotate-and-adds; square: 4095 rotations) and key-switch
    schedule given by --double-hoist, timed; the other form and schedule timed once beside it."""
    from paper_2104_03152_gb300 import inputs
    t0 = time.perf_counter()
    st = torch.cuda.Stream()
    flags = tk.TCKS_AUTO_RELIN | (tk.TCKS_DOUBLE_HOIST if args.double_hoist else 0)
    ctx = tk.Context(tk.Params(14, [60, 40, 40, 60], 2.0 ** 40), seed=inputs.SEED_KEYS, flags=flags,
                     stream=st.cuda_stream)
    ctx._torch_stream = st
    rect = args.c4_form == "rect"
    rep = [ctx.slots - C4_ROWS]
    rect_steps = list(range(1, C4_COLS)) + [C4_COLS << j for j in range(4)]
    square_steps = list(range(1, C4_ROWS))
    ctx.gen_galois_keys(rep + (rect_steps if rect else square_steps))
    M = inputs.random_matrix(C4_ROWS, C4_COLS, 7, 0.05)
    mat = ctx.matrix_encode_rect(M, level=3) if rect else ctx.matrix_encode(M, level=3)
    B = args.c4_batch
    vs = [inputs.normal_slots(C4_ROWS, 6 + 1000 * i) for i in range(B)]
    cts = []
    for i, v in enumerate(vs):
        z = np.zeros(ctx.slots)
        z[:C4_ROWS] = v
        cts.append(ctx.encrypt_values(z, 600 + i))
    ctx.synchronize()
    setup_s = time.perf_counter() - t0
    key_bytes = ctx.key_bytes()
    outs = mat.vecmat_batch(cts)  # warm-up, and the accuracy check
    err = max(float(np.max(np.abs(ctx.decrypt_values(outs[i])[:C4_COLS] - vs[i] @ M))) for i in (0, B - 1))
    torch.cuda.synchronize()
    tk.profile_start()
    per, total = timed(torch, st, lambda: mat.vecmat_batch(cts), args.c4_steps)
    tk.profile_stop()
    prof = tk.profile_read(with_ops=True)
    peak64 = tk.calibrate_butterflies(64)
    compare = {}

    def once(m, label):
        m.vecmat_batch(cts)
        _, t = timed(torch, st, lambda: m.vecmat_batch(cts), 1)
        compare[label] = {"value": B / (t / 1e3), "unit": "vectors/s"}
    if args.double_hoist:
        ctx.set_flags(tk.TCKS_AUTO_RELIN)
        once(mat, ("rectangular" if rect else "square") + ", one ModDown per rotation")
        ctx.set_flags(flags)
    if rect:  # the square form: 4095 rotations
        ctx.gen_galois_keys(square_steps)
        sq = ctx.matrix_encode(M, level=3)
        once(sq, "square" + (", ModDown once after the rotation sum" if args.double_hoist else ", one ModDown per rotation"))
        del sq
    kernels = {k: {"launches": v[0], "ms": round(v[1], 3), "gbs": round(v[2] / (v[1] / 1e3) / 1e9, 1),
                   "gbfly_s": round(v[3] / (v[1] / 1e3) / 1e9, 1),
                   "alu_frac": round(v[3] / (v[1] / 1e3) / peak64, 4)}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    return {"workload": C4_WORKLOAD, "batch": B, "value": B * args.c4_steps / (total / 1e3), "unit": "vectors/s",
            "ms_per_batch": total / args.c4_steps, "steps": args.c4_steps, "setup_s": setup_s,
            "form": ("rectangular diagonals: 255 hoisted rotations + 4 rotate-and-adds" if rect
                     else "square diagonals: 4095 hoisted rotations"),
            "galois_keys": len(rep) + len(rect_steps if rect else square_steps), "key_bytes": key_bytes,
            "max_abs_err_vs_fp64": err, "kernels": kernels, "alu_peak_bfly64_per_s": peak64,
            "schedule": "ModDown once after the rotation sum" if args.double_hoist else "one ModDown per rotation",
            "compare": compare,
            "ctx": ctx, "mat": mat, "cts": cts}


def plain_cnn(img, w):
    stride, kh = 3, 7
    conv = np.zeros((4, 8, 8))
    for k in range(4):
        ker = w["conv_w"][k].reshape(kh, kh)
        for r in range(8):
            for c in range(8):
                conv[k, r, c] = np.sum(img[stride * r:stride * r + kh, stride * c:stride * c + kh] * ker) + w["conv_b"][k]
    x = conv.reshape(-1) ** 2
    x = (w["fc1_w"] @ x + w["fc1_b"]) ** 2
    return w["fc2_w"] @ x + w["fc2_b"]


# ------------------------------------------------------------------ primitive sweep (C3) --
# Batched NTT / INTT / relinearize / rotate(1) over N in {2^13..2^16} and L in {4, 8, 16, 32} data
# primes of one chain (primes == 1 mod 2^17, data prime i of 59 - (i mod 10) bits, P of 60 bits),
# batches of ciphertexts on seeded uniform limbs, each batch a descriptor-table job list replayed from
# a CUDA graph. Rates are algorithmic: bytes = each operand read once, each result written once, each
# distinct key once; integer work = modular butterflies + modular multiply(-accumulate)s.
SWEEP_BITS = [59 - (i % 10) for i in range(32)] + [60]
SWEEP_OPS = ("ntt", "intt", "relin", "rotate")


def sweep_contexts(torch, tk, log_ns):
    from paper_2104_03152_gb300 import inputs
    primes = tk.Params(16, SWEEP_BITS, 2.0 ** 50).primes
    out = {}
    for log_n in log_ns:
        st = torch.cuda.Stream()
        c = tk.Context(tk.Params(log_n, primes=primes, scale=2.0 ** 50), seed=inputs.SEED_KEYS,
                       flags=tk.TCKS_AUTO_RELIN, stream=st.cuda_stream)
        c._torch_stream = st  # keeps the stream alive with the context
        c.gen_galois_keys([1])
        c.autotune()
        out[log_n] = c
    return out


def sweep_work(op, log_n, level, count):
    """(algorithmic bytes, algorithmic integer ops) of one job."""
    n, l = 1 << log_n, level
    bf = 0.5 * n * log_n
    if op in ("ntt", "intt"):
        limbs = 2 * count * l  # the ciphertexts' two polynomials
        return 16.0 * n * limbs, limbs * bf
    key = 8.0 * n * 2 * l * (l + 1)
    per_ct_in = (3 if op == "relin" else 2) * l * n * 8.0
    ops = count * ((l + l * l + 2 + 2 * l) * bf + (2.0 * (l + 1) * l + 2 * l) * n)
    return count * (per_ct_in + 2 * l * n * 8.0) + key, ops


def sweep_buffers(torch, ctx, op, level, count, gen):
    n = ctx.N
    polys = {"ntt": 2, "intt": 2, "relin": 3, "rotate": 2}[op]
    x = torch.empty((count, polys, level, n), dtype=torch.int64, device="cuda")
    for l in range(level):
        x[:, :, l, :] = torch.randint(0, int(ctx.primes[l]), (count, polys, n), generator=gen, device="cuda",
                                      dtype=torch.int64)
    if op in ("ntt", "intt"):
        return x, x
    return x, torch.empty((count, 2, level, n), dtype=torch.int64, device="cuda")


def sweep_job(tk, ctx, op, level, count, x, y):
    code = {"ntt": tk.JOB_NTT, "intt": tk.JOB_INTT, "relin": tk.JOB_RELIN, "rotate": tk.JOB_ROTATE}[op]
    polys = 2 * count if op in ("ntt", "intt") else count
    return (ctx, code, 1, polys, level, x.data_ptr(), y.data_ptr())


def time_graph(torch, ctx_stream, graph, reps):
    s = torch.cuda.ExternalStream(ctx_stream)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    graph.run()
    torch.cuda.synchronize()
    evs[0].record(s)
    for k in range(reps):
        graph.run()
        evs[k + 1].record(s)
    torch.cuda.synchronize()
    return sorted(evs[k].elapsed_time(evs[k + 1]) for k in range(reps))


def sweep_point(torch, tk, ctxs, entries, op, peaks, gen, reps=20, work=None):
    """entries: [(log_n, level, count)] forming one batch; returns a result dict."""
    jobs, keep, by, ops = [], [], 0.0, 0.0
    for log_n, level, count in entries:
        c = ctxs[log_n]
        x, y = sweep_buffers(torch, c, op, level, count, gen)
        keep += [x, y]
        jobs.append(sweep_job(tk, c, op, level, count, x, y))
        b, o = (work or sweep_work)(op, log_n, level, count)
        by, ops = by + b, ops + o
    graph = tk.BatchGraph(jobs)
    first = time_graph(torch, jobs[0][0].stream, graph, 1)[0]
    reps = reps if first < 100 else 5
    t = time_graph(torch, jobs[0][0].stream, graph, reps)
    ms = t[len(t) // 2]
    gbs = by / (ms * 1e-3) / 1e9
    bfly = ops / (ms * 1e-3)
    del graph, keep
    return {"op": op, "ms": round(ms, 4), "reps": reps, "algo_bytes": by, "gbs": round(gbs, 1),
            "hbm_frac": round(gbs / peaks["hbm_gbs"], 4), "gbfly_s": round(bfly / 1e9, 1),
            "alu_frac": round(bfly / peaks["bfly64_s"], 4)}


def primitive_peaks(tk):
    p = measured_peaks()
    return {"hbm_gbs": p["hbm_gbs"], "hbm_source": p["source"], "bfly64_s": tk.calibrate_butterflies(64),
            "bfly32_s": tk.calibrate_butterflies(32)}


# CPU milliseconds of the paper's unary / binary CKKSVector operation tables (appendix; N = 8192 with a
# 200-bit modulus, shapes 256 .. 16384, 2x^2 + x for polyval): another machine, context only.
OPS_SHAPES = (256, 1024, 4096, 8192, 16384)
PAPER_OPS_MS = {
    "negate": (0.07, 0.07, 0.07, 0.13, 0.26), "square": (4.29, 4.29, 4.29, 8.49, 17.16),
    "polyval": (10.55, 10.46, 10.51, 21.32, 42.68), "add": (0.08, 0.08, 0.08, 0.16, 0.31),
    "multiply": (4.45, 4.34, 4.43, 8.84, 17.75), "sub": (0.08, 0.08, 0.08, 0.15, 0.3),
    "dot": (20.15, 23.96, 28.11, 55.94, 112.36), "add_plain": (0.8, 0.86, 1.07, 2.13, 4.19),
    "multiply_plain": (1.75, 1.81, 2.03, 4.02, 7.97), "sub_plain": (0.8, 0.86, 1.08, 2.14, 4.21),
    "dot_plain": (17.37, 21.36, 25.63, 51.14, 101.82),
}


def run_ops_table(args):
    """The paper's operation tables on this GPU: each operation on an encrypted tensor of the given
    length, laid out as ceil(n / 4096) ciphertexts of up to 4096 slots (a batched CKKSTensor), through
    the public API (plain operands encoded inside the call, as the paper's timings include). Wall time
    per call with the device synchronized after it, median over --ops-reps calls."""
    import torch

    import paper_2104_03152_gb300 as tk
    from paper_2104_03152_gb300 import inputs

    tk.lib(build_if_missing=True)
    ctx = tk.Context(tk.Params(13, [60, 40, 40, 60], 2.0 ** 40), seed=inputs.SEED_KEYS,
                     flags=tk.TCKS_AUTO_RELIN | tk.TCKS_AUTO_RESCALE)
    ctx.gen_galois_keys([1 << m for m in range(12)])
    rows = {op: [] for op in PAPER_OPS_MS}
    errs = {op: 0.0 for op in PAPER_OPS_MS}
    for n in OPS_SHAPES:
        per, count = min(n, ctx.slots), (n + ctx.slots - 1) // ctx.slots
        x = np.random.default_rng(n).uniform(-1.0, 1.0, size=(per, count))
        y = np.random.default_rng(n + 1).uniform(-1.0, 1.0, size=(per, count))
        A = tk.CKKSTensor.encrypt(ctx, x, batch=True, seed=1)
        Bt = tk.CKKSTensor.encrypt(ctx, y, batch=True, seed=1 + count)
        ops = {
            "negate": (lambda: A.negate(), -x), "square": (lambda: A.square(), x * x),
            "polyval": (lambda: A.polyval([0.0, 1.0, 2.0]), 2 * x * x + x),
            "add": (lambda: A.add(Bt), x + y), "multiply": (lambda: A.mul(Bt), x * y),
            "sub": (lambda: A.sub(Bt), x - y), "dot": (lambda: A.mul(Bt).sum(), np.sum(x * y)),
            "add_plain": (lambda: A.add(y), x + y), "multiply_plain": (lambda: A.mul(y), x * y),
            "sub_plain": (lambda: A.sub(y), x - y), "dot_plain": (lambda: A.mul(y).sum(), np.sum(x * y)),
        }
        for op, (fn, ref) in ops.items():
            for _ in range(args.warmup):
                fn()
            ctx.synchronize()
            ts = []
            for _ in range(args.ops_reps):
                t0 = time.perf_counter()
                r = fn()
                ctx.synchronize()
                ts.append((time.perf_counter() - t0) * 1e3)
            rows[op].append(statistics.median(ts))
            errs[op] = max(errs[op], float(np.max(np.abs(r.decrypt() - ref))))
        del A, Bt
        torch.cuda.synchronize()
    for op, ms in rows.items():
        print(json.dumps({"table": "ckksvector_ops", "op": op, "shapes": list(OPS_SHAPES), "gpu_ms": ms,
                          "paper_cpu_ms": list(PAPER_OPS_MS[op]), "max_abs_err": errs[op],
                          "config": {"log_n": 13, "bits": [60, 40, 40, 60], "scale": "2^40",
                                     "slots_per_ciphertext": 4096, "reps": args.ops_reps,
                                     "timing": "wall time of the API call + device synchronize, median"}}))


def run_sweep(args):
    import torch
    import paper_2104_03152_gb300 as tk
    tk.lib(build_if_missing=True)
    torch.cuda.set_device(0)
    peaks = primitive_peaks(tk)
    print(json.dumps({"sweep_peaks": peaks}), flush=True)
    log_ns = [int(x) for x in args.sweep_log_n.split(",")]
    ctxs = sweep_contexts(torch, tk, log_ns)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    batches = [int(b) for b in args.sweep_batches.split(",")]
    levels = [int(x) for x in args.sweep_L.split(",")]
    ops = args.sweep_ops.split(",")
    for log_n in log_ns:
        for L in levels:
            for B in batches:
                for op in ops:
                    r = sweep_point(torch, tk, ctxs, [(log_n, L, B)], op, peaks, gen)
                    r.update({"log_n": log_n, "L": L, "batch": B})
                    print(json.dumps(r), flush=True)
                torch.cuda.empty_cache()
    # mixed batches: every ciphertext draws (N, L) uniformly; one job per (N, L) group, one graph
    rng = np.random.default_rng(5)
    for B in [b for b in batches if b > 1 and args.sweep_mixed]:
        draws = [(int(rng.choice(log_ns)), int(rng.choice(levels))) for _ in range(B)]
        groups = {}
        for d in draws:
            groups[d] = groups.get(d, 0) + 1
        entries = [(ln, L, cnt) for (ln, L), cnt in sorted(groups.items())]
        for op in ops:
            r = sweep_point(torch, tk, ctxs, entries, op, peaks, gen)
            r.update({"mixed": True, "batch": B, "groups": len(entries)})
            print(json.dumps(r), flush=True)
        torch.cuda.empty_cache()


HYB_SPECIAL, HYB_ALPHA = 8, 8  # hybrid key switching at the sweep's largest shape: 4 digits of 8 primes, 8 special


def ks_transforms(level: int, alpha: int = 1, special: int = 1) -> int:
    """Length-N transforms of one key switch at `level`: the INTT of the input, the NTT of every converted
    digit limb, the INTT of the special limbs and the NTT of the ModDown's conversions (2 components)."""
    dn = -(-level // alpha)
    return level + (dn * (level + special) - level) + 2 * special + 2 * level


def hybrid_contexts(torch, tk, log_n: int, special: int, alpha: int):
    from paper_2104_03152_gb300 import inputs
    bits = SWEEP_BITS[:-1] + [60] * special
    primes = tk.Params(log_n, bits, 2.0 ** 50).primes
    st = torch.cuda.Stream()
    c = tk.Context(tk.Params(log_n, primes=primes, scale=2.0 ** 50, n_special=special, alpha=alpha),
                   seed=inputs.SEED_KEYS, flags=tk.TCKS_AUTO_RELIN, stream=st.cuda_stream)
    c._torch_stream = st
    c.gen_galois_keys([1])
    return {log_n: c}


def sweep_work_hybrid(op, log_n, level, count, special, alpha):
    """(algorithmic bytes, algorithmic integer ops) of one hybrid job: inputs and outputs once, the key
    (dnum digits x 2 x (level + K) limbs) once; transforms plus conversion and inner-product products."""
    n, l = 1 << log_n, level
    bf = 0.5 * n * log_n
    dn = -(-l // alpha)
    key = 8.0 * n * dn * 2 * (l + special)
    per_ct_in = (3 if op == "relin" else 2) * l * n * 8.0
    conv = (dn * (l + special) - l) * alpha + 2 * l * special  # base-conversion products per coefficient
    inner = 2 * dn * (l + special)  # inner-product products per coefficient
    ops = count * (ks_transforms(l, alpha, special) * bf + (conv + inner + 2 * l) * n)
    return count * (per_ct_in + 2 * l * n * 8.0) + key, ops


def primitives_summary(torch, tk):
    """NTT and key-switch rates at the largest sweep shape (N = 2^16, L = 32, 64 ciphertexts), with the
    one-prime key switch and with hybrid key switching (4 digits of 8 primes, 8 special primes)."""
    peaks = primitive_peaks(tk)
    ctxs = sweep_contexts(torch, tk, [16])
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    out = {"shape": "N=2^16, L=32 data primes (50-60-bit), 64 ciphertexts per batch, CUDA-graph replay",
           "peaks": {"hbm_gbs": peaks["hbm_gbs"], "bfly64_per_s": peaks["bfly64_s"], "bfly32_per_s": peaks["bfly32_s"]},
           "transforms_per_key_switch": {"one_prime": ks_transforms(32),
                                         "hybrid": ks_transforms(32, HYB_ALPHA, HYB_SPECIAL)}}
    for op in SWEEP_OPS:
        out[op] = sweep_point(torch, tk, ctxs, [(16, 32, 64)], op, peaks, gen)
    del ctxs
    torch.cuda.empty_cache()
    hyb = hybrid_contexts(torch, tk, 16, HYB_SPECIAL, HYB_ALPHA)
    for op in ("relin", "rotate"):
        r = sweep_point(torch, tk, hyb, [(16, 32, 64)], op, peaks, gen,
                        work=lambda o, ln, lv, cnt: sweep_work_hybrid(o, ln, lv, cnt, HYB_SPECIAL, HYB_ALPHA))
        r["key_switching"] = f"hybrid: {-(-32 // HYB_ALPHA)} digits of {HYB_ALPHA} primes, {HYB_SPECIAL} special primes"
        out[op + "_hybrid"] = r
    del hyb
    torch.cuda.empty_cache()
    return out


CONV_LABEL = {
    "shared+pack+fold": ("hoisted sums, the pack masks folded into the baby-step diagonals over the input's "
                         "rotations (one diagonal-method sum and one ModDown per request for the 4 kernels), one "
                         "giant-step sum per request"),
    "shared+pack": ("hoisted sums, baby steps over the input's rotations shared by the 4 kernels, channels packed "
                    "before one giant-step sum per request"),
    "shared": "hoisted sums, baby steps over the input's rotations shared by the 4 kernels (one ModUp per request)",
    "hoist": "two hoisted rotation sums per kernel (7 baby + 7 giant steps, one ModDown each)",
    "chain": "rotate-and-add chain (6 key switches)",
}


def conv_form(args) -> str:
    if not args.conv_hoist:
        return "chain"
    if not args.conv_shared:
        return "hoist"
    if not args.conv_pack:
        return "shared"
    return "shared+pack+fold" if args.conv_fold else "shared+pack"


# ------------------------------------------------------------------------------ CPU oracle --
def oracle_setup(rect: bool = True, conv_hoist: bool = True, conv_shared: bool = True, conv_pack: bool = True,
                 fold: bool = True):
    import oracle
    from paper_2104_03152_gb300 import inputs

    o = oracle.OracleCKKS(LOG_N, BITS, SCALE, key_seed=inputs.SEED_KEYS).keygen()
    shared, pack = conv_hoist and conv_shared, conv_hoist and conv_shared and conv_pack
    for st, lv in oracle.cnn_galois_steps(o, rect=rect, conv_hoist=conv_hoist, conv_shared=shared,
                                          pack_first=pack).items():
        o.gen_galois_key(st, lv)
    w = oracle.CNNWeights(**inputs.cnn_weights(SEED_W))
    enc = oracle.cnn_encode(o, w, rect=rect, conv_hoist=conv_hoist, conv_shared=shared, pack_first=pack,
                            fold=pack and fold)
    img = inputs.mnist_like_image(SEED_IMG)
    v, _ = oracle.OracleCKKS.im2col(img, 7, 7, 3, o.slots)
    ct = o.encrypt_values(v, SEED_ENC)
    return oracle, o, w, enc, ct


def time_oracle(n_steps: int, warmup: int, double_hoist: bool = True, single_thread_steps: int = 0,
                rect: bool = True, conv_hoist: bool = True, conv_shared: bool = True, conv_pack: bool = True,
                merged: bool = True, fold: bool = True):
    """Oracle CNN inferences on the host cores (same schedule as the GPU arm); optionally also
    single-threaded ones. Returns (times, cores, single-thread times)."""
    oracle, o, w, enc, ct = oracle_setup(rect, conv_hoist, conv_shared, conv_pack, fold)
    for _ in range(warmup):
        oracle.cnn_forward(o, ct, w, enc, double_hoist=double_hoist, merged=merged)
    times = []
    for _ in range(n_steps):
        t0 = time.perf_counter()
        oracle.cnn_forward(o, ct, w, enc, double_hoist=double_hoist, merged=merged)
        times.append(time.perf_counter() - t0)
    cores = oracle.lib().orc_max_threads()
    single = []
    if single_thread_steps:
        oracle.lib().orc_set_threads(1)
        for _ in range(single_thread_steps):
            t0 = time.perf_counter()
            oracle.cnn_forward(o, ct, w, enc, double_hoist=double_hoist, merged=merged)
            single.append(time.perf_counter() - t0)
        oracle.lib().orc_set_threads(cores)
    return times, cores, single


def run_reference(args, world, rank):
    if rank != 0:
        return
    steps, warmup = args.steps, args.warmup
    # bound the run: at most ~3 minutes of oracle inferences
    times, cores, _ = time_oracle(steps, warmup, bool(args.double_hoist), 0, args.fc_form == "rect",
                                  bool(args.conv_hoist), bool(args.conv_shared), bool(args.conv_pack),
                                  bool(args.merged_rescale), bool(args.conv_fold))
    total = sum(times)
    value = steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "inferences/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * total / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": "cpu oracle",
                       "vecmat_schedule": ("ModDown once after each rotation sum (double hoisting)"
                                           if args.double_hoist else "one ModDown per rotation"),
                       "fc_form": "rectangular diagonals" if args.fc_form == "rect" else "square diagonals",
                       "conv_form": CONV_LABEL[conv_form(args)]},
            "cpu_baseline": {"value": value, "unit": "inferences/s", "cores": cores, "kind": "oracle",
                             "sample": f"{steps} full inferences (forward only; keys and weights prepared outside)"},
            "e2e": {"value": value, "unit": "inferences/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------ main --
PROFILE_CASES = {
    # name: (log_n, data primes, op, ciphertexts, special primes, alpha)
    "ntt-n16-l32": (16, 32, "ntt", 8, 1, 1),
    "intt-n16-l32": (16, 32, "intt", 8, 1, 1),
    "relin-n16-l32": (16, 32, "relin", 2, 1, 1),
    "rotate-n16-l32": (16, 32, "rotate", 2, 1, 1),
    "relin-hyb-n16-l32": (16, 32, "relin", 2, HYB_SPECIAL, HYB_ALPHA),
    "rotate-hyb-n16-l32": (16, 32, "rotate", 2, HYB_SPECIAL, HYB_ALPHA),
}


def run_profile_case(args):
    """One small case for a profiler: a primitive job at the sweep's largest shape (PROFILE_CASES), or
    'cnn-b<B>' (the bench's CNN layout on B requests), run --warmup times, then --steps times inside
    the NVTX range 'case', eagerly (no graph), so that `ncu --nvtx --nvtx-include case/ -k ...` takes
    exactly the launches of the case."""
    import torch

    import paper_2104_03152_gb300 as tk
    tk.lib(build_if_missing=True)
    torch.cuda.set_device(0)
    name = args.profile_case
    if name.startswith("cnn-b"):
        B = int(name[5:])
        tk_, ctx, model, cts, stream, imgs, w = gpu_setup(torch, B, True, True, True, True, True, True, True)
        d_in = torch.empty((B, 2, cts[0].level, ctx.N), dtype=torch.int64, device="cuda")
        for i, c in enumerate(cts):
            d_in[i].copy_(torch.from_numpy(c.export().view(np.int64)))
        d_out = torch.empty((B, 2, cts[0].level - 6, ctx.N), dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        step = lambda: model.forward_device(d_in.data_ptr(), B, d_out.data_ptr())
        sync = ctx.synchronize
    else:
        log_n, L, op, count, special, alpha = PROFILE_CASES[name]
        from paper_2104_03152_gb300 import inputs
        bits = SWEEP_BITS[:L] + [60] * special
        primes = tk.Params(log_n, bits, 2.0 ** 50).primes
        ctx = tk.Context(tk.Params(log_n, primes=primes, scale=2.0 ** 50, n_special=special, alpha=alpha),
                         seed=inputs.SEED_KEYS, flags=tk.TCKS_AUTO_RELIN)
        ctx.gen_galois_keys([1])
        gen = torch.Generator(device="cuda")
        gen.manual_seed(5)
        x, y = sweep_buffers(torch, ctx, op, L, count, gen)
        job = sweep_job(tk, ctx, op, L, count, x, y)
        step = lambda: tk.batch_run([job])
        sync = ctx.synchronize
    for _ in range(args.warmup):
        step()
    sync()
    torch.cuda.nvtx.range_push("case")
    for _ in range(args.steps):
        step()
    sync()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile_case": name, "steps": args.steps, "warmup": args.warmup}))


def served_vs_plain(serving):
    """The first trace's served and plain throughput and p99 latency, side by side."""
    if not serving or not serving.get("traces"):
        return None
    t = serving["traces"][0]
    sv, pl = t["served"], t["plain"]
    return {"offered_rate": t["offered_rate"], "served_throughput": sv["throughput"], "served_p50_ms": sv["p50_ms"],
            "served_p99_ms": sv["p99_ms"], "plain_throughput": pl["throughput"], "plain_p50_ms": pl["p50_ms"],
            "plain_p99_ms": pl["p99_ms"], "unit": "requests/s, ms (arrival -> result on the host)",
            "measured_seconds": t["seconds"], "requests": t["requests"],
            "plain_requests": pl.get("trace_requests")}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=2, help="oracle inferences timed for cpu_baseline")
    ap.add_argument("--batch", type=int, default=256, help="requests per step (the batched schedule)")
    ap.add_argument("--serve-batch", type=int, default=64, help="largest batch the serving loop forms per stage")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="measured length of the Poisson serving trace (0: skip)")
    ap.add_argument("--serve-warmup", type=float, default=1.0,
                    help="seconds of trace served before the measured part (not counted)")
    ap.add_argument("--serve-rate", default="2000",
                    help="offered requests/s of the serving traces (comma-separated; one trace each)")
    ap.add_argument("--cnn-clients", type=int, default=8, help="CNN clients of the trace, each with its own keys")
    ap.add_argument("--vm-clients", type=int, default=2,
                    help="vector x matrix clients of the trace, each with its own keys")
    ap.add_argument("--sweep", action="store_true", help="print the batched primitive sweep (JSON lines) and exit")
    ap.add_argument("--ops-table", action="store_true",
                    help="print the paper's CKKSVector operation tables measured here (JSON lines) and exit")
    ap.add_argument("--ops-reps", type=int, default=20)
    ap.add_argument("--tune-cache", type=int, default=0,
                    help="reuse / record the network autotuner's choice in a JSON file in the temp directory")
    ap.add_argument("--profile-case", default="",
                    help="run one small case for a profiler (" + ", ".join(PROFILE_CASES) + ", cnn-b<B>) and exit")
    ap.add_argument("--sweep-batches", default="1,8,64,512", help="ciphertexts per batch in the sweep")
    ap.add_argument("--sweep-log-n", default="13,14,15,16", help="log2 N values of the sweep")
    ap.add_argument("--sweep-L", default="4,8,16,32", help="data-prime counts of the sweep")
    ap.add_argument("--sweep-ops", default=",".join(SWEEP_OPS), help="ops of the sweep")
    ap.add_argument("--sweep-mixed", type=int, default=1, help="also run the mixed (N, L) batches")
    ap.add_argument("--primitives", type=int, default=1, help="add the NTT / key-switch rates at N=2^16, L=32")
    ap.add_argument("--fc-form", default="rect", choices=["rect", "square"],
                    help="diagonal form of the CNN's fully connected layers")
    ap.add_argument("--conv-hoist", type=int, default=1,
                    help="the convolution sums as hoisted baby-step giant-step rotation sums (1) or a chain (0)")
    ap.add_argument("--conv-shared", type=int, default=1,
                    help="with --conv-hoist 1: the baby steps over the input's rotations, shared by the kernels")
    ap.add_argument("--conv-pack", type=int, default=1,
                    help="with --conv-shared 1: pack the channels before one giant-step sum per request")
    ap.add_argument("--conv-fold", type=int, default=1,
                    help="fold the pack masks into the shared baby-step diagonals (one sum per request)")
    ap.add_argument("--merged-rescale", type=int, default=1,
                    help="take every ModDown that precedes a rescale and the rescale as one rounding")
    ap.add_argument("--double-hoist", type=int, default=1,
                    help="vector x matrix products take the ModDown once after the rotation sum (1) or per rotation (0)")
    ap.add_argument("--c4", type=int, default=1, help="time the 4096x256 vector x matrix workload (64 vectors)")
    ap.add_argument("--c4-batch", type=int, default=64)
    ap.add_argument("--c4-form", default="rect", choices=["rect", "square"],
                    help="diagonal form of the 4096x256 matrix (rect: 260 rotations, square: 4096)")
    ap.add_argument("--c4-steps", type=int, default=3)
    ap.add_argument("--serve-mix", type=float, default=0.3, help="share of vector x matrix requests in the trace")
    ap.add_argument("--plain-requests", type=int, default=0,
                    help="requests at the start of each trace replayed through the plain path (0: the whole trace)")
    args = ap.parse_args()
    if args.sweep:
        run_sweep(args)
        return
    if args.ops_table:
        run_ops_table(args)
        return
    if args.profile_case:
        run_profile_case(args)
        return
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    r = run_gpu(args, world, rank, local)
    if rank != 0:
        return
    peaks = measured_peaks()
    B = args.batch
    ms_per_step = r["total_ms"] / args.steps
    value = job_value(world, B, args.steps, r["total_ms"])
    # dominant kernel family by device time
    prof = r["prof"]
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    name, (nl, ms, by, ops) = dom
    hbm_ach = by / (ms / 1e3) / 1e9
    alu_ach = ops / (ms / 1e3) / 1e9
    # sums of products (the double-hoisted accumulation) against the rate of the kernel's own form at each
    # launch's level (tcks_calibrate_dh_macs), transforms against the measured butterfly rate
    mac_kernel = name == "vecmat_dh_acc"
    shapes = None
    if mac_kernel and r["dh_records"]:
        t_min, shapes = 0.0, {}
        for tag, rms, rops in r["dh_records"]:
            ell, outs, unit = tag & 0xFF, (tag >> 8) & 0xFF, (tag >> 16) & 1
            t_min += rops / r["dh_peaks"][ell]
            key = f"level {ell}, {outs} output{'s' if outs > 1 else ''}{', unit diagonals' if unit else ''}"
            sh = shapes.setdefault(key, {"launches": 0, "ms": 0.0, "ops": 0.0, "ceiling_gmacs": r["dh_peaks"][ell] / 1e9})
            sh["launches"] += 1
            sh["ms"] += rms
            sh["ops"] += rops
        for sh in shapes.values():
            sh["achieved_gmacs"] = sh["ops"] / (sh["ms"] / 1e3) / 1e9
            sh["frac"] = sh["achieved_gmacs"] / sh["ceiling_gmacs"]
        alu_peak = ops / t_min / 1e9  # the work-weighted ceiling of the family's launches
    else:
        alu_peak = (r["mac_peak"] if mac_kernel else r["bfly_peak"]) / 1e9
    traffic = ncu_traffic(name, {"batch": B, "fc_form": args.fc_form, "conv_hoist": args.conv_hoist,
                                 "conv_form": conv_form(args), "merged_rescale": args.merged_rescale,
                                 "double_hoist": args.double_hoist})
    hbm = {"achieved": hbm_ach, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": hbm_ach / peaks["hbm_gbs"],
           "peak_source": peaks["source"]}
    alu = {"achieved": alu_ach, "peak": alu_peak, "unit": "Gmac/s" if mac_kernel else "Gbfly/s",
           "frac": alu_ach / alu_peak if alu_peak else None,
           "peak_source": ("measured: tcks_calibrate_dh_macs(level) on this GPU -- the kernel's own form (unreduced "
                           "key-switch sums, carry-chain diagonal products, one logic op per load) from registers, "
                           "at each launch's level, weighted by each launch's work" if shapes else
                           f"measured: tcks_calibrate_{'macs' if mac_kernel else 'butterflies'}({r['word']}) on this "
                           "GPU, registers only"),
           "per_shape": shapes,
           "generic_mac_peak_gmacs": r["mac_peak"] / 1e9 if mac_kernel else None}
    bound = "alu" if alu["frac"] and alu["frac"] > hbm["frac"] else "hbm"
    top = alu if bound == "alu" else hbm
    roofline = {"kernel": name, "bound": bound, "achieved": top["achieved"], "peak": top["peak"], "unit": top["unit"],
                "frac": top["frac"], "peak_source": top["peak_source"], "traffic": traffic,
                "hbm": hbm, "alu": alu, "launches": nl, "algo_bytes_per_launch": by / nl,
                "algo_ops_per_launch": ops / nl, "avg_launch_us": 1e3 * ms / nl,
                "ops_unit": ("modular product-accumulates (key-switch sums and diagonal products)" if mac_kernel
                             else "modular butterflies + modular multiply(-accumulate)s")}
    kernels = {k: {"launches": v[0], "ms": round(v[1], 4), "share": round(v[1] / sum(x[1] for x in prof.values()), 4),
                   "gbs": round(v[2] / (v[1] / 1e3) / 1e9, 1), "gbfly_s": round(v[3] / (v[1] / 1e3) / 1e9, 1)}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    per = sorted(r["per_step"])
    # CPU baseline: the oracle on the host cores, bounded sample
    if args.cpu_sample > 0:
        times, cores, single = time_oracle(args.cpu_sample, 0, bool(args.double_hoist), 1, args.fc_form == "rect",
                                           bool(args.conv_hoist), bool(args.conv_shared), bool(args.conv_pack),
                                           bool(args.merged_rescale), bool(args.conv_fold))
        cpu_val = len(times) / sum(times)
    else:
        times, cores, cpu_val, single = [], 0, None, []
    line = {
        "metric": METRIC, "value": value, "unit": "inferences/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": f"u{r['word']}", "data": "synthetic",
        "dtype_note": ("exact residues modulo primes below 2^31 held in 32-bit words" if r["word"] == 32
                       else "exact residues in 64-bit words"),
        "config": {"workload": WORKLOAD, "batch": B, "galois_keys": r["galois_keys"],
                   "vecmat_schedule": ("ModDown once after each rotation sum (double hoisting)" if args.double_hoist
                                       else "one ModDown per rotation"),
                   "fc_form": ("rectangular diagonals: FC1 63 + 2 rotations, FC2 15 + 2 (no replication)"
                               if args.fc_form == "rect" else "square diagonals: FC1 255 rotations, FC2 63"),
                   "conv_form": CONV_LABEL[conv_form(args)],
                   "l2": "inputs larger than L2 (Galois keys ~0.75 GB + key-switch scratch streamed per step)",
                   "launch_shape": r["tune"],
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "latency_ms": {"p50": per[len(per) // 2], "p99": per[min(len(per) - 1, int(0.99 * len(per)))],
                       "mode": f"batched step of {B} requests (each request completes with its batch)"},
        "plain": {"value": 1e3 / r["plain_ms"], "unit": "inferences/s", "ms_per_inference": r["plain_ms"],
                  "p99_ms": sorted(r["plain_times"])[min(len(r["plain_times"]) - 1, int(0.99 * len(r["plain_times"])))],
                  "mode": "one request at a time"},
        "accuracy": {"max_abs_err_vs_fp64": r["max_err"], "scale": "2^26"},
        "roofline": roofline, "kernels": kernels,
        "cpu_baseline": {"value": cpu_val, "unit": "inferences/s", "cores": cores, "kind": "oracle",
                         "sample": f"{len(times)} full CNN inferences of this workload (forward only, same "
                                   "vector x matrix schedule)",
                         "single_thread": {"value": len(single) / sum(single) if single else None, "cores": 1,
                                           "sample": f"{len(single)} inference(s)"}},
        "e2e": {"value": world * B * r["e2e_steps"] / r["wire_s"], "unit": "inferences/s",
                "h2d_bytes_per_step": r["wire_h2d"], "d2h_bytes_per_step": r["wire_d2h"],
                "api": "tcks_cnn_pipe_submit / tcks_cnn_pipe_wait (the pipelined tcks_cnn_forward_wire, two "
                       "batches in flight): seeded serialized inputs in (%d bytes each, c0 bit-packed + the "
                       "seed of c1, plus its 8-byte seed copied to the device), serialized outputs out (%d bytes "
                       "each); unpacking, c1 from its seed and packing on the device, inside the timed region"
                       % r["wire_sizes"]},
        "e2e_unpipelined": {"value": world * B * r["e2e_steps"] / r["wire_sync_s"], "unit": "inferences/s",
                            "h2d_bytes_per_step": r["wire_h2d"], "d2h_bytes_per_step": r["wire_d2h"],
                            "api": "tcks_cnn_forward_wire, one synchronous call per batch"},
        "e2e_limbs": {"value": world * B * r["e2e_steps"] / r["e2e_s"], "unit": "inferences/s",
                      "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"],
                      "api": "tcks_cnn_forward_host: 64-bit limbs in and out"},
        "served_vs_plain": served_vs_plain(r["serving"]),
        "serving": r["serving"],
        "primitives": r["primitives"],
        "compare": r["single"],
        "vecmat_4096x256": r["c4"],
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
