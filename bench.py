"""Throughput of the multislice loss + object/probe gradient on GB300.

One step = one full evaluation of the hot path through the C-ABI
(``ptycho_loss_grad``): the slice chain of every position (forward model,
amplitude residual, exact adjoint), the tiled object-gradient accumulation,
the probe-gradient and FP64 loss reductions.  Metric: probe positions per
second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config 1|2|3|5|6] [--impl reference]

Inputs are synthetic (seeded) and resident in HBM when the timed region
starts; the L2 is flushed (512 MiB write) between timed steps, outside the
per-step CUDA events.  The default line is the 576-position multislice
workload; after it, the same line carries the 16632-position PbTiO3-shaped
workload (``paper_shaped``) and the 32 batched uneven problems under one CUDA
graph per iteration (``batched``), and ``parity`` gives the timed path's
errors against the FP64 oracle on 48 of the positions.  ``e2e`` repeats the measurement through the public
Python API with host (pinned) inputs and host results, copies included (the
call goes to ``ptycho_loss_grad_host``, which uploads the later positions'
intensities while the first chain wave runs).
``--impl reference`` times the FP64 CPU oracle on the host cores instead.
Under torchrun (N > 1) every rank runs an independent replica of the
workload (the evaluation has no data exchange between GPUs); rank 0
prints the line with the max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "probe-positions/s for loss+object/probe gradient; % of HBM/tensor roofline"
UNIT = "positions/s"
FP32_LANES_PER_SM = 128  # FP32 FMA lanes per Blackwell SM (4 partitions x 32)


# --------------------------------------------------------------------------
# workload
# --------------------------------------------------------------------------

def workload_for(config_id: int):
    from paper_2205_06327_gb300 import synth
    return synth.workload(config_id)


def start_object(wl, seed: int = 7):
    """A reconstruction iterate near the truth (seeded perturbation)."""
    from paper_2205_06327_gb300 import synth
    g = synth.rng(seed)
    return wl.obj * np.exp(0.1j * g.standard_normal(wl.obj.shape))


def flops_per_position(M: int, S: int) -> float:
    """Algorithmic FP32 flops of one position's chain + gradient patch.

    FFTs: (2S-1) forward + (2S-1) adjoint 2-D transforms at 5 M^2 log2(M^2)
    each.  Elementwise (per pixel): S transmissions and S-1 propagator
    multiplies forward, the same adjoint (6 flops per complex multiply), the
    residual (10) and the object-gradient patch conj(psi) g (8 with the add).
    """
    fft = 5.0 * M * M * math.log2(M * M)
    n_fft = 4 * S - 2
    elem = M * M * (6 * S + 6 * (S - 1) + 10 + 6 * S + 6 * (S - 1) + 8 * S)
    return n_fft * fft + elem


def chain_flops_per_position(M: int, S: int) -> float:
    """Flops of the slice-chain kernel alone (everything but the patch products)."""
    return flops_per_position(M, S) - 8.0 * S * M * M


def tensor_flops_per_position(M: int, S: int) -> float:
    """Tensor-core flops of one position on the BF16-split path: 2S transforms
    (S-1 propagations and the far field, forward and adjoint), each two
    M x M x M complex products, each four real products of three BF16 terms."""
    return 2 * S * 2 * 4 * 3 * 2.0 * M ** 3


def peaks_tensor() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"bf16_tflops": d.get("bf16_tflops", 1900.0), "src": "measured (cuBLAS bf16 burst)"}
    return {"bf16_tflops": 1900.0, "src": "fallback"}


def hbm_bytes_per_evaluation(wl) -> float:
    """Minimum bytes the method moves per evaluation: intensities once, object
    once, object gradient once, probe and its gradient."""
    return (wl.N * wl.M * wl.M * 4 + 2 * wl.S * wl.H * wl.W * 8 + 2 * wl.M * wl.M * 8)


# --------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline): process pool, spawn context
# --------------------------------------------------------------------------

_ORC_STATE = {}


def _as_c64(a):
    """The complex64 values the GPU receives, widened again for the oracle."""
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


def _oracle_init(config_id: int):
    from oracle import ptycho_oracle as orc
    wl = workload_for(config_id)
    _ORC_STATE["wl"] = wl
    _ORC_STATE["probe"] = _as_c64(wl.probe)
    _ORC_STATE["obj"] = _as_c64(start_object(wl))
    _ORC_STATE["h"] = orc.fresnel_propagator(wl.M, wl.lambda_A, wl.dz_A, wl.pixel_A)


def _oracle_task(args):
    from oracle import ptycho_oracle as orc
    idx, I = args
    wl = _ORC_STATE["wl"]
    L, gO, gP = orc.loss_grad(_ORC_STATE["probe"], _ORC_STATE["obj"], wl.pos[idx], I.astype(np.float64),
                              _ORC_STATE["h"])
    # return only the bounding box of the windows touched
    y0, x0 = wl.pos[idx].min(0)
    y1, x1 = wl.pos[idx].max(0) + wl.M
    return L, (int(y0), int(x0)), gO[:, y0:y1, x0:x1], gP


class OraclePool:
    def __init__(self, config_id: int, cores: int):
        self.cores = cores
        ctx = mp.get_context("spawn")
        self.pool = ctx.Pool(cores, initializer=_oracle_init, initargs=(config_id,))
        self.pool.map(abs, range(cores))  # wait for the workers

    def loss_grad(self, wl, idx: np.ndarray, I: np.ndarray):
        """One oracle loss+gradient over positions idx (I rows for them):
        (F, dF/dO, dF/dP, wall seconds)."""
        parts = np.array_split(np.asarray(idx), min(self.cores, len(idx)))
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_task, [(p, I[p]) for p in parts if len(p)])
        L = 0.0
        gO = np.zeros((wl.S, wl.H, wl.W), complex)
        gP = np.zeros((wl.M, wl.M), complex)
        for l, (y0, x0), g, p in res:
            L += l
            gO[:, y0:y0 + g.shape[1], x0:x0 + g.shape[2]] += g
            gP += p
        return L, gO, gP, time.perf_counter() - t0

    def evaluate(self, wl, idx: np.ndarray, I: np.ndarray) -> float:
        """One oracle loss+gradient over positions idx; returns wall seconds."""
        return self.loss_grad(wl, idx, I)[3]

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_model() -> str:
    """The host CPU's model name (lscpu), else the machine type."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip() + f" ({platform.machine()})"
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def cpu_sample_indices(wl, n_sample: int) -> np.ndarray:
    if n_sample >= wl.N:
        return np.arange(wl.N)
    return np.linspace(0, wl.N - 1, n_sample).round().astype(np.int64)


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, path: str | None):
        self.path = path
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
            if self.path:
                with open(self.path, "w") as f:
                    f.write(self.FIELDS + "\n" + "\n".join(self.lines) + "\n")
        return False

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------
# distributed helpers (replicas; host logic covered by gloo tests)
# --------------------------------------------------------------------------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value: float, world: int, device=None) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None and device.type == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# --------------------------------------------------------------------------
# arms
# --------------------------------------------------------------------------

CHAIN_SOURCES = {"fp32": ("chain_kernels.cu", "chain_body.inc", "fft2d.cuh"), "bf16x3": ("chain_tc.cu", "tc_bf16.cuh"),
                 "fp16x3": ("chain_tc.cu", "tc_bf16.cuh")}


# every kernel of one evaluation: the chain, the reductions, and the host code that launches them
STEP_SOURCES = {p: CHAIN_SOURCES[p] + ("reduce_kernels.cu", "ptycho_api.cu") for p in CHAIN_SOURCES}


def chain_source_hash(precision: str, names=None) -> str:
    import hashlib
    h = hashlib.sha256()
    for name in (names or CHAIN_SOURCES[precision]):
        with open(os.path.join(ROOT, "paper_2205_06327_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_step_traffic_per_position(precision: str, M: int, S: int):
    """DRAM bytes per position of a whole evaluation (every kernel of one step,
    ncu, profiles/traffic.json), or None if any of those sources changed."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(f"step_{precision}_M{M}_S{S}")
    if not e or e.get("source_hash") != chain_source_hash(precision, STEP_SOURCES[precision]):
        return None
    return float(e["dram_bytes_per_position"])


def measured_traffic_per_position(precision: str, M: int, S: int):
    """DRAM bytes per position of the chain kernel from the committed ncu capture
    (profiles/traffic.json), or None if the kernel changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(f"{precision}_M{M}_S{S}")
    if not e or e.get("source_hash") != chain_source_hash(precision):
        return None
    return float(e["dram_bytes_per_position"])


def peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "src": "measured"}
    return {"hbm_gbs": 6800.0, "src": "fallback"}


def run_reference(args, world, rank):
    """FP64 CPU oracle on the host cores: each step one bounded sample."""
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    wl = workload_for(args.config)
    pool = OraclePool(args.config, cores)
    # measured intensities for the sample from the oracle itself (noise-free, scaled)
    from oracle import ptycho_oracle as orc
    idx = cpu_sample_indices(wl, args.cpu_sample)
    h = orc.fresnel_propagator(wl.M, wl.lambda_A, wl.dz_A, wl.pixel_A)
    I = np.zeros((wl.N, wl.M, wl.M), np.float32)
    I[idx] = orc.intensities(wl.probe, wl.obj, wl.pos[idx], h).astype(np.float32)
    for _ in range(args.warmup):
        pool.evaluate(wl, idx, I)
    times = [pool.evaluate(wl, idx, I) for _ in range(args.steps)]
    pool.close()
    t = float(np.mean(times))
    v = len(idx) / t
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "positions_per_step": int(len(idx)), "M": wl.M, "S": wl.S,
                   "object": [wl.H, wl.W]},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "cpu": cpu_model(), "kind": "oracle",
                         "sample": f"{len(idx)} of {wl.N} positions per step (loss + object/probe gradient)"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def fp32_peak(device, sm_mhz) -> tuple[float, str]:
    """FP32 ALU peak (TFLOP/s) of the device that ran: its SM count times 128
    FMA lanes times 2 flops at the median SM clock sampled in the timed region
    (the nominal maximum clock if no sample was taken)."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mhz, how = sm_mhz, "median SM clock sampled in the timed region"
    if not mhz:
        mhz, how = 2070.0, "nominal maximum clock (no clock samples)"
    return (sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12,
            f"derived: {sms} SMs (device property) x {FP32_LANES_PER_SM} FP32 lanes x 2 flops x {mhz:.0f} MHz "
            f"({how})")


def measure_workload(wl, config_id, args, device, world, rank, local, ckpt_every, steps, warmup, clocks_path):
    """Time `steps` evaluations of workload wl (after `warmup`) through
    ptycho_loss_grad with inputs resident in HBM.  Returns the measurement and
    the device tensors (for the end-to-end and parity legs)."""
    import torch

    from paper_2205_06327_gb300 import api

    obj0 = start_object(wl)
    geom = api.Geometry(wl.M, wl.S, wl.H, wl.W, wl.N, wl.lambda_A, wl.dz_A, wl.pixel_A)
    tile = tuple(int(v) for v in args.tile.split("x")) if args.tile else (0, 0)
    ws = int(args.workspace_mb) << 20
    plan = api.Plan(geom, device, async_check=True, timing=True, tile=tile, ckpt_every=ckpt_every,
                    precision=args.precision, workspace_bytes=ws)
    pos = torch.from_numpy(wl.pos).to(device)
    probe = torch.from_numpy(wl.probe.astype(np.complex64)).to(device)
    obj_true = torch.from_numpy(wl.obj.astype(np.complex64)).to(device)
    obj = torch.from_numpy(obj0.astype(np.complex64)).to(device)
    # measurements: forward model at the truth (GPU), Poisson counts (seeded)
    _, I = plan.forward(pos, probe, obj_true, want_psi=False, want_intensity=True)
    del obj_true
    if wl.counts is not None:
        gen = torch.Generator(device=device)
        gen.manual_seed(1000 + config_id)
        I = torch.poisson(I, generator=gen)
    if config_id == 3 and not args.tile:
        # The gradient is accumulated per tile; the tile shape only changes the
        # speed (results are bit-identical), so the 8 x 8 tessellation of the
        # workload competes with smaller tiles and the fastest is kept.
        from paper_2205_06327_gb300 import autotune
        tess = ((wl.H + 7) // 8, (wl.W + 7) // 8)
        tile = autotune.tune_tile(geom, pos, probe, obj, I, device, precision=args.precision,
                                  candidates=(tess, (32, 32), (16, 64), (32, 64), (64, 32)), reps=1,
                                  use_cache=False, ckpt_every=ckpt_every)
        plan.close()
        plan = api.Plan(geom, device, async_check=True, timing=True, tile=tile, ckpt_every=ckpt_every,
                        precision=args.precision, workspace_bytes=ws)
    gO = torch.empty((wl.S, wl.H, wl.W), dtype=torch.complex64, device=device)
    gP = torch.empty((wl.M, wl.M), dtype=torch.complex64, device=device)
    loss = torch.empty((), dtype=torch.float64, device=device)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=device)
    stream = torch.cuda.current_stream(device)
    lib, h, sh = plan.lib, plan._h, stream.cuda_stream

    def step():
        rc = lib.ptycho_loss_grad(h, pos.data_ptr(), probe.data_ptr(), obj.data_ptr(), I.data_ptr(),
                                  loss.data_ptr(), gO.data_ptr(), gP.data_ptr(), sh)
        if rc:
            from paper_2205_06327_gb300._lib import check
            check(rc)

    for _ in range(warmup):
        flush.fill_(1)
        step()
    torch.cuda.synchronize(device)
    plan.timing(reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    clocks = ClockSampler(local, clocks_path)
    barrier(world, device)
    torch.cuda.synchronize(device)
    wall0 = time.perf_counter()
    with clocks:
        for k in range(steps):
            flush.fill_(k & 0xff)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize(device)
    wall = time.perf_counter() - wall0
    barrier(world, device)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tm = plan.timing(reset=True)
    plan.status()
    del flush
    t_step = float(np.mean(step_ms)) / 1e3
    t_max = reduce_max(t_step, world, device)
    csum = clocks.summary()

    # roofline of the dominant kernel (slice chain): FP32 ALU bound, or the
    # tensor pipe for the split-precision transforms.  Per launch: the
    # kernel's events on the launching stream cover all chain launches.
    chain_ms = tm["chain_ms"] / max(tm["chain_launches"], 1)
    chain_pos = tm["chain_positions"] / max(tm["chain_launches"], 1)
    # recompute mode: K launches share one evaluation's chain work
    chain_work = tm["chain_positions"] / max(wl.N * steps, 1)
    if args.precision != "fp32":
        chain_flops = tensor_flops_per_position(wl.M, wl.S) * chain_pos / chain_work
        pk_t = peaks_tensor()
        peak_tflops = pk_t["bf16_tflops"]
        bound, peak_src = "tensor", pk_t["src"]
    else:
        chain_flops = chain_flops_per_position(wl.M, wl.S) * chain_pos / chain_work
        peak_tflops, peak_src = fp32_peak(device, csum["sm_mhz"])
        bound = "alu"
    achieved = chain_flops / (chain_ms / 1e3) / 1e12
    tpp = measured_traffic_per_position(args.precision, wl.M, wl.S) if not ckpt_every else None
    traffic = tpp * chain_pos if tpp is not None else None
    pk = peaks()
    # accumulation, per launch: the workspace arrays it reads (conj(psi) and
    # g_phi per slice, or the finished patches in recompute mode) for the
    # launch's positions and slices, and the object gradient (written by a
    # step's first launch of each slice, read and rewritten by the later ones)
    n_acc = max(tm["accum_launches"], 1)
    accum_ms = tm["accum_ms"] / n_acc
    per_step = n_acc / steps
    if ckpt_every:  # one launch per (chunk, segment): the segment's slices, the chunk's positions
        n_seg = -(-wl.S // ckpt_every)
        n_chunks = per_step / n_seg
        sl, acc_pos, arrays = wl.S / n_seg, wl.N / n_chunks, 1.0
        grad_bytes = sl * wl.H * wl.W * 8 * (1.0 + 2.0 * (n_chunks - 1)) / n_chunks
    else:           # one or two launches per chunk (full waves, tail): every slice
        sl, acc_pos, arrays = wl.S, wl.N / per_step, 2.0
        grad_bytes = wl.S * wl.H * wl.W * 8 * (1.0 + 2.0 * (per_step - 1)) / per_step
    accum_bytes = arrays * acc_pos * sl * wl.M * wl.M * 8 + grad_bytes
    launches_per_step = tm["launches"] / steps
    meas = {
        "value": world * wl.N / t_max, "t_max": t_max, "step_ms": step_ms, "wall": wall, "tile": tile,
        "csum": csum, "plan_chunk": plan.chunk, "workspace_bytes": plan.workspace_bytes,
        "launches_per_step": launches_per_step, "geom": geom,
        "roofline": {"bound": bound, "kernel": "k_chain (slice chain, gradient mode)"
                     if args.precision == "fp32" else "k_chain_tc (split DFT products, gradient mode)",
                     "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": traffic,
                     "peak_src": peak_src,
                     "kernel_ms": chain_ms, "kernel_share": tm["chain_ms"] / max(sum(step_ms), 1e-9)},
        "hbm_kernels": {"accum_obj_grad": {"ms": accum_ms, "bytes": accum_bytes,
                                           "gbs": accum_bytes / (accum_ms / 1e3) / 1e9 if accum_ms else None,
                                           "frac": (accum_bytes / (accum_ms / 1e3) / 1e9) / pk["hbm_gbs"]
                                           if accum_ms else None, "peak_src": pk["src"]}},
        "path_bound_ms": max(flops_per_position(wl.M, wl.S) * wl.N / (peak_tflops * 1e12),
                             hbm_bytes_per_evaluation(wl) / (pk["hbm_gbs"] * 1e9)) * 1e3,
        "tensors": (pos, probe, obj, I, gO, gP),
    }
    plan.close()
    return meas


def step_traffic(wl, args):
    """DRAM bytes per position of a whole evaluation against the method's
    algorithmic bytes (intensities, object, object gradient once each)."""
    if args.ckpt_every or args.positions or args.order != "raster":
        return None
    b = measured_step_traffic_per_position(args.precision, wl.M, wl.S)
    if b is None:
        return None
    alg = hbm_bytes_per_evaluation(wl) / wl.N
    return {"dram_bytes_per_position": b, "algorithmic_bytes_per_position": alg, "ratio": b / alg,
            "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum over every kernel of one "
                      "evaluation (profiles/traffic.json)"}


def parity_sample(wl, args, device, tile, ckpt_every, tensors, pool, k=48):
    """Relative errors of the timed path against the FP64 oracle on k positions
    spread over the scan (outside the timed region): the same kernels, launch
    configuration and inputs, restricted to those positions."""
    import torch

    from paper_2205_06327_gb300 import api
    pos, probe, obj, I = tensors[:4]
    idx = cpu_sample_indices(wl, k)
    sel = torch.from_numpy(idx).to(device)
    g = api.Geometry(wl.M, wl.S, wl.H, wl.W, len(idx), wl.lambda_A, wl.dz_A, wl.pixel_A)
    plan = api.Plan(g, device, async_check=True, tile=tile, ckpt_every=ckpt_every, precision=args.precision,
                    workspace_bytes=int(args.workspace_mb) << 20)
    L, gO, gP = plan.loss_grad(pos[sel].contiguous(), probe, obj, I[sel].contiguous())
    torch.cuda.synchronize(device)
    plan.close()
    Lr, gOr, gPr, _ = pool.loss_grad(wl, idx, I.cpu().numpy())
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    return {"positions": int(len(idx)), "loss": abs(float(L) - Lr) / abs(Lr),
            "grad_obj": rel(gO.cpu().numpy(), gOr), "grad_probe": rel(gP.cpu().numpy(), gPr),
            "reference": "FP64 oracle on the complex64 inputs, same positions",
            "bar": "rel-L2 1e-5 (FP32) / 2e-4 (split precisions)"}


def run_gpu(args, world, rank, local, pool):
    import torch

    from paper_2205_06327_gb300 import api

    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)

    wl = workload_for(args.config)
    if args.positions:
        wl.pos = wl.pos[: args.positions]
    if args.order == "shuffled":
        wl.pos = wl.pos[np.random.default_rng(12345).permutation(len(wl.pos))]
    if args.ckpt_every is None:  # the PbTiO3-shaped and paper-scale workloads recompute waves in
        # the adjoint: ceil(sqrt(S)) checkpoints, so every 5 of 30 and every 10 of 100 slices
        args.ckpt_every = {3: 5, 6: 10}.get(args.config, 0)
    m = measure_workload(wl, args.config, args, device, world, rank, local, args.ckpt_every, args.steps,
                         args.warmup, f"{args.clocks_csv}.r{rank}.csv" if args.clocks_csv else None)
    pos, probe, obj, I, gO, gP = m["tensors"]
    geom, tile = m["geom"], m["tile"]

    # end to end through the public API: pinned host inputs, host results
    e2e = None
    if not args.no_e2e:
        hp = {k: v.cpu().pin_memory() for k, v in (("pos", pos), ("probe", probe), ("obj", obj), ("I", I))}
        h2d = sum(v.numel() * v.element_size() for v in hp.values())
        d2h = 8 + gO.numel() * 8 + gP.numel() * 8
        eplan = api.Plan(geom, device, async_check=True, tile=tile, ckpt_every=args.ckpt_every,
                         precision=args.precision, workspace_bytes=int(args.workspace_mb) << 20)
        flush = torch.empty(512 << 20, dtype=torch.uint8, device=device)
        # warm-up as in the timed loop: the previous results stay alive while
        # the next call runs, so the pinned result buffers are all allocated
        for _ in range(3):
            L, go, gp = eplan.loss_grad(hp["pos"], hp["probe"], hp["obj"], hp["I"])
        torch.cuda.synchronize(device)
        ts = []
        for _ in range(max(3, args.steps // 2)):
            flush.fill_(3)
            torch.cuda.synchronize(device)
            t0 = time.perf_counter()
            L, go, gp = eplan.loss_grad(hp["pos"], hp["probe"], hp["obj"], hp["I"])
            _ = float(L)
            ts.append(time.perf_counter() - t0)
        eplan.close()
        del flush
        print("e2e ms per evaluation: " + " ".join(f"{1e3 * t:.3f}" for t in ts), file=sys.stderr)
        te = reduce_max(float(np.mean(ts)), world, device)
        e2e = {"value": world * wl.N / te, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    cpu, parity = None, None
    if pool is not None and rank == 0:
        idx = cpu_sample_indices(wl, args.cpu_sample)
        I_host = I.cpu().numpy()
        pool.evaluate(wl, idx[: min(len(idx), pool.cores)], I_host)  # warm the workers
        t_cpu = pool.evaluate(wl, idx, I_host)
        cpu = {"value": len(idx) / t_cpu, "unit": UNIT, "cores": pool.cores, "cpu": cpu_model(), "kind": "oracle",
               "sample": f"{len(idx)} of {wl.N} positions, one loss + object/probe gradient evaluation "
                         f"(FP64 NumPy, process pool)"}
        if not args.positions and args.order == "raster":
            parity = parity_sample(wl, args, device, tile, args.ckpt_every, m["tensors"], pool)
    del pos, probe, obj, I, gO, gP, m["tensors"]

    # the workload closest to the paper (16632 positions, Table I's count),
    # timed after the headline measurement
    paper_shaped = None
    if args.config == 2 and not args.no_paper_shaped and not args.positions:
        w3 = workload_for(3)
        m3 = measure_workload(w3, 3, args, device, world, rank, local, 5, max(3, args.steps // 4), 3, None)
        del m3["tensors"]
        paper_shaped = {"workload": w3.name, "positions": w3.N, "M": w3.M, "S": w3.S, "object": [w3.H, w3.W],
                        "value": m3["value"], "unit": UNIT, "ms_per_step": m3["t_max"] * 1e3,
                        "steps": max(3, args.steps // 4), "ckpt_every": 5, "tiles": list(m3["tile"]),
                        "workspace_bytes": m3["workspace_bytes"], "chunk": m3["plan_chunk"],
                        "roofline": m3["roofline"], "hbm_kernels": m3["hbm_kernels"],
                        "gpu_launches_per_step": m3["launches_per_step"],
                        "clocks": {"sm_mhz": m3["csum"]["sm_mhz"], "reasons": m3["csum"]["reasons"]}}

    # the batched workload (32 uneven problems, one CUDA graph per iteration),
    # timed over fewer iterations than its own run
    batched = None
    if args.config == 2 and not args.no_batched and not args.positions:
        mb = measure_multi(args, device, world, local, 10, 3)
        batched = {"workload": f"{mb['problems']} uneven problems (windows 64-256, 1-24 slices), one CUDA "
                               "graph per gradient-descent iteration",
                   "value": mb["value"], "unit": UNIT, "ms_per_step": mb["ms_per_step"],
                   "iterations": mb["iterations"], "positions_per_iteration": mb["positions_per_iteration"],
                   "gpu_launches_per_step": mb["gpu_launches_per_step"], "tiles": mb["tiles"],
                   "clocks": {"sm_mhz": mb["csum"]["sm_mhz"], "reasons": mb["csum"]["reasons"]}}

    csum = m["csum"]
    line = {
        "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["t_max"] * 1e3,
        "ms_per_step_median": float(np.median(m["step_ms"])), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "bf16x3": "bf16x3+f32", "fp16x3": "f16x3+f32"}[args.precision],
        "data": "synthetic",
        "config": {"workload": wl.name, "positions": wl.N, "M": wl.M, "S": wl.S, "object": [wl.H, wl.W],
                   "tiles": list(tile) if tile != (0, 0) else [32, 32],
                   "l2": "flushed between timed steps (512 MiB write, outside the step events)",
                   "replicas": world, "wall_s": m["wall"], "ckpt_every": args.ckpt_every, "order": args.order,
                   "workspace_bytes": m["workspace_bytes"], "chunk": m["plan_chunk"]},
        "roofline": m["roofline"],
        "hbm_kernels": m["hbm_kernels"],
        "path_bound_ms": m["path_bound_ms"],
        "step_traffic": step_traffic(wl, args),
        "e2e": e2e, "cpu_baseline": cpu, "parity": parity,
        "gpu_launches": int(round(m["launches_per_step"] * args.steps)),
        "gpu_launches_per_step": m["launches_per_step"],
        "clocks": {"sm_mhz": csum["sm_mhz"], "sm_max_mhz": csum["sm_max_mhz"], "reasons": csum["reasons"]},
        "paper_shaped": paper_shaped,
        "batched": batched,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def measure_multi(args, device, world, local, iterations, warmup):
    """Batched uneven reconstructions: the 32 seeded problem shapes, each
    advanced by fixed-step gradient descent, all problems of one iteration in a
    single captured CUDA graph; the accumulation tile is tuned per window size."""
    import torch

    from paper_2205_06327_gb300 import api, autotune, synth
    from paper_2205_06327_gb300.multi import MultiProblem, Problem, supported

    shapes = synth.multi_problem_shapes()
    probs, skipped = [], []
    windows = {int(x) for x in args.windows.split(",")} if args.windows else None
    for p, (M, S, ny, nx, step) in enumerate(shapes):
        if windows is not None and M not in windows:
            continue
        if args.problems and len(probs) >= args.problems:
            break
        if not supported(M, args.precision):
            skipped.append(M)
            continue
        wl = synth.workload_random(M, S, ny, nx, step, seed=synth.MULTI_SEED_BASE + p)
        g = api.Geometry(wl.M, wl.S, wl.H, wl.W, wl.N, wl.lambda_A, wl.dz_A, wl.pixel_A)
        pos = torch.from_numpy(wl.pos).to(device)
        probe = torch.from_numpy(wl.probe.astype(np.complex64)).to(device)
        truth = torch.from_numpy(wl.obj.astype(np.complex64)).to(device)
        plan = api.Plan(g, device, async_check=True, precision=args.precision)
        _, I = plan.forward(pos, probe, truth, want_psi=False, want_intensity=True)
        plan.close()
        obj = torch.from_numpy(start_object(wl, seed=p).astype(np.complex64)).to(device)
        probs.append(Problem(g, pos, probe, obj, I * 1.05))
        del truth
    tiles = {}
    for pr in probs:  # one tuning run per window size, on that class's first problem
        if pr.geom.M not in tiles:
            tiles[pr.geom.M] = autotune.tune_tile(pr.geom, pr.pos, pr.probe, pr.obj, pr.meas, device,
                                                  precision=args.precision, use_cache=False)
        pr.tile = tiles[pr.geom.M]
    mp = MultiProblem(probs, device, precision=args.precision)
    for pl in mp.plans:
        pl.timing(reset=True)
    mp.capture(1e-3, 1e-6, warmup=warmup)
    # the library counts the kernels each call enqueues: warm-up iterations
    # plus the captured one; a replay launches the captured iteration's kernels
    launches_per_iter = sum(pl.timing(reset=True)["launches"] for pl in mp.plans) / (warmup + 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(device)
    barrier(world, device)
    torch.cuda.synchronize(device)
    clocks = ClockSampler(local, None)
    with clocks:
        e0.record(stream)
        mp.run(iterations)
        e1.record(stream)
        torch.cuda.synchronize(device)
    barrier(world, device)
    mp.check_status()
    t = e0.elapsed_time(e1) / 1e3
    t_max = reduce_max(t, world, device)
    per_it = mp.positions_per_iteration
    out = {"value": world * per_it * iterations / t_max, "ms_per_step": t_max / iterations * 1e3,
           "iterations": iterations, "problems": len(probs), "skipped_windows": skipped,
           "positions_per_iteration": per_it, "tiles": {str(k): list(v) for k, v in tiles.items()},
           "gpu_launches_per_step": launches_per_iter, "csum": clocks.summary(),
           "final_loss_sum": float(mp.loss.sum().item())}
    mp.close()
    return out


def run_multi(args, world, rank, local):
    import torch
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    m = measure_multi(args, device, world, local, args.iterations, args.warmup)
    csum = m["csum"]
    line = {
        "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": m["iterations"],
        "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "bf16x3": "bf16x3+f32", "fp16x3": "f16x3+f32"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"{m['problems']} uneven problems of the 32 seeded shapes (windows 64-256, "
                               "1-24 slices), one CUDA graph per gradient-descent iteration"
                               + (f", windows {args.windows} only" if args.windows else ""),
                   "problems": m["problems"], "skipped_windows": m["skipped_windows"],
                   "positions_per_iteration": m["positions_per_iteration"], "iterations": m["iterations"],
                   "tiles": m["tiles"],
                   "l2": "inputs larger than L2 in aggregate; no flush between graph replays"},
        "gpu_launches": int(round(m["gpu_launches_per_step"] * m["iterations"])),
        "gpu_launches_per_step": m["gpu_launches_per_step"],
        "clocks": {"sm_mhz": csum["sm_mhz"], "sm_max_mhz": csum["sm_max_mhz"], "reasons": csum["reasons"]},
        "final_loss_sum": m["final_loss_sum"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 5, 6],
                    help="workload: 1 single slice, 2 multislice (default), 3 PbTiO3-shaped, 5 batched uneven, "
                         "6 the paper's per-position shape (1024^2 window, 100 slices) on 8 positions")
    ap.add_argument("--iterations", type=int, default=50, help="gradient-descent iterations (workload 5)")
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=576)
    ap.add_argument("--positions", type=int, default=0, help="first N positions only (profiling cases)")
    ap.add_argument("--order", default="raster", choices=["raster", "shuffled"],
                    help="GPU legs: positions in the workload's raster order, or a seeded random permutation "
                         "(the library uses the caller's order; this measures what the order costs)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16x3", "fp16x3"],
                    help="bf16x3 / fp16x3: 2-D transforms as hi/lo split DFT products on the tensor cores")
    ap.add_argument("--tile", default="",
                    help="object-gradient accumulation tile HxW (e.g. 16x64; default: the library's, "
                         "tuned for workload 3)")
    ap.add_argument("--workspace-mb", type=int, default=0,
                    help="cap on the plan's workspace in MiB (0: the library's default, 8 GiB); the "
                         "positions run in chunks that fit it")
    ap.add_argument("--ckpt-every", type=int, default=None,
                    help="recompute mode: keep a wave checkpoint every L slices (0 = keep all)")
    ap.add_argument("--windows", default="",
                    help="workload 5: only the problems with these windows, e.g. 192,256 (profiling cases)")
    ap.add_argument("--problems", type=int, default=0, help="workload 5: the first N problems only")
    ap.add_argument("--clocks-csv", default="",
                    help="also keep the raw nvidia-smi clock samples of the timed region (<path>.r<rank>.csv)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-paper-shaped", action="store_true",
                    help="skip the second measurement, of the 16632-position PbTiO3-shaped workload")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the third measurement, of the 32 batched uneven problems (10 iterations)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.config == 5:
        return run_multi(args, world, rank, local)
    pool = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # spawn the oracle's workers before the first CUDA call (no more than
        # the sample has positions: each worker holds the workload)
        n_pos = 8 if args.config == 6 else args.cpu_sample  # workload 6 has 8 positions
        pool = OraclePool(args.config, max(1, min(os.cpu_count() or 1, n_pos, args.cpu_sample)))
    try:
        return run_gpu(args, world, rank, local, pool)
    finally:
        if pool is not None:
            pool.close()


if __name__ == "__main__":
    sys.exit(main())
