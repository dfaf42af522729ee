#!/usr/bin/env python
"""Throughput of the RNS-CKKS evaluation core on GB300.

One step = one pass of the hot path over one batch at N = 2^16:
  * 64 ciphertext pairs with 24 ciphertext primes (q0 ~ 2^61, 23 x ~2^55),
    8 special primes, dnum = 3: HMult + relinearise + rescale (batched);
  * every one of the 64 inputs rotated by 2^0 .. 2^14 (hoisted: 960 rotations);
  * 16 exhausted ciphertexts bootstrapped (2^15 slots, 25 + 9 primes, 16 levels).
`value` is HMult+relin(+rescale)/s over the multiply phase of the timed steps
(device time, CUDA events on the library's stream); rotations/s and
bootstraps/s come from the other two phases.  Inputs (over 3 GB of
ciphertexts per step) exceed L2, so no flush.

--impl reference times the CPU oracle on the host cores instead (bounded
sample: one HMult+relin+rescale of one ciphertext pair per step).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic_inputs as si  # noqa: E402

METRIC = "HMult+relin/s and bootstraps/s at N=2^16 on 1 GB300, plain vs batched TC form"
UNIT = "HMult+relin/s"


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def peaks():
    """(HBM GB/s, dense bf16 TFLOP/s sustained, "measured" | "fallback")."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("bf16_tflops_sustained", p["bf16_tflops"])), "measured"
    return 6800.0, 1700.0, "fallback"


def traffic_table():
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"ckks_bench_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx.append(float(parts[1]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[4:8]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- ranks
# Weak scaling: the N ranks process N independent batches (their own messages
# and encryption randomness), so the data path has no exchange; the only
# collectives are the barriers around the timed region and the max-over-ranks
# of the timings.
def shard_seeds(rank):
    """Seeds of one rank's inputs: messages and encryption randomness of the
    products and rotations, of the bootstraps, of the RE-Block step and of
    the uneven batch."""
    return {"mul": 100 + rank, "boot": 300 + rank, "reboot": 400 + rank, "uneven": 500 + rank}


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of per-rank timings (a float list) over all ranks."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_rates(world, pairs, rotations_per_ct, boots, steps, mul_ms, rot_ms, boot_ms):
    """Whole-job rates: every rank's units over the slowest rank's time."""
    return {"hmult_per_s": world * pairs * steps / (mul_ms / 1e3),
            "rotations_per_s": world * pairs * rotations_per_ct * steps / (rot_ms / 1e3),
            "bootstraps_per_s": world * boots * steps / (boot_ms / 1e3)}


# ---------------------------------------------------------------- oracle arm
class OracleSample:
    """The CPU oracle on one ciphertext pair of the workload (keys and inputs
    prepared once, untimed); time() runs one HMult+relin+rescale with the
    merged ModDown-rescale, the computation the GPU arm times."""

    def __init__(self, w, seed=0):
        import oracle
        self.orc = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
        self.orc.keygen(1)
        level = len(w.q_bits) - 1
        scale = 2.0 ** w.log2_scale
        z = si.messages(seed, 2, w.slots)
        self.cts = [self.orc.encrypt(self.orc.pt_from_int(self.orc.encode(z[i], scale), level), level, scale,
                                     10 + i) for i in range(2)]
        self.threads = _env_int("OMP_NUM_THREADS", os.cpu_count() or 1)

    def time(self) -> float:
        t0 = time.perf_counter()
        self.orc.mul_relin_rescale(self.cts[0], self.cts[1])
        return time.perf_counter() - t0

    def time_rotation(self, k: int = 1) -> float:
        """One rotation of the same ciphertext (its key generated untimed)."""
        self.orc.gen_rotation_keys([k])
        t0 = time.perf_counter()
        self.orc.rotate(self.cts[0], k)
        return time.perf_counter() - t0


def run_reference(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    w = si.PLAIN
    sample = OracleSample(w)
    threads = sample.threads
    for _ in range(min(args.warmup, 1)):
        sample.time()
    times = [sample.time() for _ in range(args.steps)]
    v = 1.0 / float(np.mean(times))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": config_of(w, w.batch, args.form),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "per step: 1 HMult+relin+rescale of 1 ciphertext pair at N=2^16, L=24 "
                                       "(1/64 of the batch), CPU oracle (128-bit % arithmetic, OpenMP over limbs)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


FORM_NAMES = {"uint64": "uint64 CUDA-core basis conversion",
              "tensor": "byte-split basis conversion on tcgen05 tensor cores",
              "fused": "uint64 basis conversion fused with the NTTs' column passes (one kernel per column tile)"}


def config_of(w, batch, form):
    return {"workload": w.name, "log_n": w.log_n, "n_q": len(w.q_bits), "n_p": len(w.p_bits), "dnum": w.dnum,
            "log2_scale": w.log2_scale, "batch_pairs": batch, "rotations_per_ct": len(w.rot_steps),
            "form": FORM_NAMES[form], "rescale": "ModDown and rescale merged into one basis conversion",
            "l2": "inputs over 400 MB per step > 126 MB L2; no flush"}


# ---------------------------------------------------------------- GPU arm
# Roofline model (the roofs of each form): every kernel class is measured
# against HBM and against the compute pipe its form runs on -- the integer
# pipe for the uint64 CUDA-core kernels (the measured rate of the production
# instruction sequence, ckks_alu_peaks), the tensor pipe for the byte-split
# basis conversion (fp16 MMA at the measured dense bf16 rate).  The binding
# roof is the one with the larger fraction (the tighter lower bound on time).
# Units are the library profiler's: a limb of N words, except the basis
# conversions (one source-target limb pair of one polynomial) and the
# bootstrap's plaintext MAC and linear combination (one limb of N words moved
# to or from HBM).
ALU_UNITS = {"mac_per_s": "64x64->128 MAC/s", "bfly_fwd_loose_per_s": "Shoup butterflies/s",
             "bfly_fwd_strict_per_s": "Shoup butterflies/s", "bfly_inv_approx_per_s": "Shoup butterflies/s",
             "bfly_inv_exact_per_s": "Shoup butterflies/s"}


def ip_digits(ks_hist, w):
    """Average digit count of the key inner products, weighted by their
    extended limbs (from the key-switch histogram); the top level's count
    when no histogram is given."""
    nq = len(w.q_bits)
    alpha = -(-nq // w.dnum)
    num = den = 0
    for lvl, cnt in enumerate(ks_hist or []):
        if cnt:
            ext = lvl + 1 + len(w.p_bits)
            num += cnt * ext * (-(-(lvl + 1) // alpha))
            den += cnt * ext
    return num / den if den else -(-nq // alpha)


def kernel_work(name, units, w, ndig, prof):  # noqa: C901
    """(HBM bytes, [(integer ops, roof key)], tensor flops) of `units` units of
    kernel class `name`."""
    n = 1 << w.log_n
    lh = w.log_n - 8
    hbm_words = {"ntt_fwd_pass_a": 2, "ntt_fwd_pass_b": 2, "ntt_inv_pass_a": 2, "ntt_inv_pass_b": 2,
                 "ntt_fwd_cluster": 2, "ntt_fwd_pass_b_finish": 3,
                 "automorph": 2, "tensor": 7, "ks_moddown_combine": 8, "ks_inner_product": ndig + 2,
                 "boot_mac_ext": 1, "boot_lincomb": 1, "bconv": None, "bconv_tc": None}.get(name)
    alu, tensor = [], None
    if name.startswith("ntt_"):
        # the one-pass cluster form runs all log2 N stages per limb
        per_limb = (n // 2) * (lh if name.endswith("pass_a") else w.log_n if name.endswith("cluster") else 8)
        if name.startswith("ntt_fwd"):
            # strict limbs are counted for every forward transform that runs the column stages
            fwd_limbs = prof.get("ntt_fwd_pass_a", (0, 0, 0))[2] + prof.get("ntt_fwd_cluster", (0, 0, 0))[2]
            f = prof.get("ntt_fwd_strict_limbs", (0, 0, 0))[2] / max(1, fwd_limbs)
            alu = [(units * (1 - f) * per_limb, "bfly_fwd_loose_per_s"), (units * f * per_limb, "bfly_fwd_strict_per_s")]
        else:
            f = prof.get("ntt_inv_exact_limbs", (0, 0, 0))[2] / max(1, prof.get("ntt_inv_pass_a", (0, 0, 1))[2])
            alu = [(units * (1 - f) * per_limb, "bfly_inv_approx_per_s"), (units * f * per_limb, "bfly_inv_exact_per_s")]
    elif name == "bconv":
        alu = [(units * n, "mac_per_s")]
    elif name == "conv_fused":
        # the conversion's MACs plus the column stages of the transforms around it
        g = lambda k: prof.get(k, (0, 0, 0))[2]  # noqa: E731
        src, dst, strict = g("fused_src_limbs"), g("fused_dst_limbs"), g("fused_dst_strict_limbs")
        half = (n // 2) * lh
        alu = [(units * n, "mac_per_s"), (src * half, "bfly_inv_approx_per_s"),
               ((dst - strict) * half, "bfly_fwd_loose_per_s"), (strict * half, "bfly_fwd_strict_per_s")]
        return 8 * n * (src + dst), alu, None
    elif name == "ks_inner_product":
        alu = [(units * 2 * ndig * n, "mac_per_s")]
    elif name == "boot_mac_ext":
        # the launches' multiply-accumulates, counted by the library (all launches of the class)
        alu = [(prof.get("boot_mac_ext_macs", (0, 0, 0))[2] * (units / max(1, prof.get(name, (0, 0, 1))[2])),
                "mac_per_s")]
    if name == "bconv_tc":
        tensor = units * n * 64 * 2  # 8 x 8 byte products per coefficient and pair, 2 flops each
    if name in ("bconv", "bconv_tc"):
        # the sources once, the targets once: per pair that is at least 8 N / sources
        # + 8 N / targets; the launch's pairs come as 8 x 24 (ModUp) or 9 x 23 (merged)
        hbm = units * 8 * n * (1 / 24 + 1 / 8)
    else:
        hbm = hbm_words * 8 * n * units if hbm_words is not None else None
    if name == "ntt_fwd_pass_b_finish":
        # the transformed limb, the accumulator limb and the output limb, plus a
        # base limb where the finish adds one (counted by the library)
        base = prof.get("finish_base_limbs", (0, 0, 0))[2] * (units / max(1, prof.get(name, (0, 0, 1))[2]))
        hbm += 8 * n * base
    return hbm, alu, tensor


def part(prof, ks_hist, w):
    """One context's profile: (profile, workload, inner-product digits)."""
    return (prof, w, ip_digits(ks_hist, w))


def class_work(parts, name):
    """Device ms, launches, units and algorithmic work of one kernel class,
    summed over the contexts' profiles."""
    ms = nl = units = 0
    hbm, alu, tensor = 0.0, [], 0.0
    have_hbm = have_tc = False
    for prof, w, ndig in parts:
        m, l, u = prof.get(name, (0.0, 0, 0))
        if not l:
            continue
        ms, nl, units = ms + m, nl + l, units + u
        h, a, t = kernel_work(name, u, w, ndig, prof)
        if h is not None:
            hbm, have_hbm = hbm + h, True
        alu += a
        if t is not None:
            tensor, have_tc = tensor + t, True
    return ms, nl, units, (hbm if have_hbm else None), alu, (tensor if have_tc else None)


def timed_classes(parts):
    out = {}
    for prof, _, _ in parts:
        for k, v in prof.items():
            if v[1]:
                out[k] = out.get(k, 0.0) + v[0]
    return out


def roofline(parts, hbm_peak, peak_kind, alu_peaks, tensor_peak=None, name=None):
    """Roofs of one kernel class (default: the one with the most device time in
    the timed region): HBM plus the compute pipe of its form."""
    classes = timed_classes(parts)
    total = sum(classes.values())
    if name is None:
        name = max(classes.items(), key=lambda kv: kv[1])[0]
    ms, nlaunch, units, hbm, alu, tensor = class_work(parts, name)
    if not nlaunch:
        return None
    sec = ms / 1e3
    roofs = {}
    if hbm is not None:
        a = hbm / sec / 1e9
        roofs["hbm"] = {"achieved": a, "peak": hbm_peak, "unit": "GB/s", "frac": a / hbm_peak,
                        "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json copy bandwidth)",
                        "algorithmic_per_launch": hbm / nlaunch}
    if tensor is not None and tensor_peak:
        a = tensor / sec / 1e12
        roofs["tensor"] = {"achieved": a, "peak": tensor_peak, "unit": "TFLOP/s", "frac": a / tensor_peak,
                           "peak_source": f"{peak_kind} bf16_tflops_sustained (fp16 runs at the bf16 rate)",
                           "algorithmic_per_launch": tensor / nlaunch}
    if alu and alu_peaks:
        t_min = sum(ops / alu_peaks[key] for ops, key in alu)
        ops = sum(o for o, _ in alu)
        keys = sorted({k for o, k in alu if o})
        roofs["alu"] = {"achieved": ops / sec / 1e12, "peak": ops / t_min / 1e12 if t_min else None,
                        "unit": "T " + ALU_UNITS[keys[0] if keys else alu[0][1]], "frac": t_min / sec,
                        "peak_source": "measured on this GPU by ckks_alu_peaks: register-only kernels running "
                                       "the production instruction sequence (" + ", ".join(keys) + ")",
                        "algorithmic_per_launch": ops / nlaunch}
    if not roofs:
        return None
    bound = max(roofs, key=lambda k: roofs[k]["frac"])
    best = dict(roofs[bound])
    tr = traffic_table().get(name)
    traffic = (tr["dram_bytes_per_unit"] * units / nlaunch
               if tr and tr.get("valid") and tr.get("dram_bytes_per_unit") else None)
    best.update({"bound": bound, "kernel": name, "avg_launch_us": ms / nlaunch * 1e3, "launches": nlaunch,
                 "share_of_timed_device_ms": ms / total if total else None, "traffic": traffic,
                 "traffic_source": "profiles/traffic.json (ncu dram__bytes_read.sum + dram__bytes_write.sum "
                                   "per unit x units per launch)" if traffic else None,
                 "roofs": {k: {kk: vv for kk, vv in v.items() if kk != "peak_source"} for k, v in roofs.items()}})
    return best


def kernel_rooflines(parts, hbm_peak, peak_kind, alu_peaks, tensor_peak):
    """Every kernel class with a work model, by share of device time: the
    binding roof and the fraction of each roof."""
    classes = timed_classes(parts)
    total = sum(classes.values())
    out = {}
    for name, ms in sorted(classes.items(), key=lambda kv: -kv[1]):
        r = roofline(parts, hbm_peak, peak_kind, alu_peaks, tensor_peak, name=name)
        nl = class_work(parts, name)[1]
        out[name] = {"share": round(ms / total, 4), "avg_launch_us": round(ms / nl * 1e3, 2),
                     "bound": r["bound"] if r else None, "frac": round(r["frac"], 4) if r else None,
                     "fracs": {k: round(v["frac"], 4) for k, v in r["roofs"].items()} if r else None}
    return out


def op_roofline(parts, ops, seconds, hbm_peak, alu_peaks, tensor_peak, bytes_per_op):
    """Op-level roofline of one phase: `ops` operations took `seconds` of device
    time.  HBM: bytes_per_op (the method's own minimum) at the copy bandwidth.
    Compute: every kernel class's algorithmic integer and tensor work in the
    phase (profiler units) at its measured roof, summed."""
    t_alu = t_tc = 0.0
    for name in timed_classes(parts):
        _, _, _, _, alu, tensor = class_work(parts, name)
        t_alu += sum(o / alu_peaks[k] for o, k in alu)
        if tensor:
            t_tc += tensor / (tensor_peak * 1e12)
    rate = ops / seconds
    hbm_frac = bytes_per_op * rate / (hbm_peak * 1e9)
    comp_frac = (t_alu + t_tc) / seconds
    return {"ops_per_s": rate, "hbm": {"bytes_per_op": bytes_per_op, "achieved_gbs": bytes_per_op * rate / 1e9,
                                       "frac": hbm_frac},
            "compute": {"integer_pipe_s_per_op": t_alu / ops, "tensor_pipe_s_per_op": t_tc / ops,
                        "frac": comp_frac},
            "bound": "hbm" if hbm_frac >= comp_frac else "compute", "frac": max(hbm_frac, comp_frac)}


def hmult_bytes(w, batch):
    """Fused lower bound of one HMult+relin+rescale: read both inputs, the
    relinearisation key once per batch, write the product one level down."""
    n, L, K = 1 << w.log_n, len(w.q_bits), len(w.p_bits)
    alpha = -(-L // w.dnum)
    ndig = -(-L // alpha)
    return 8 * n * (2 * 2 * L + ndig * 2 * (L + K) / batch + 2 * (L - 1))


def rotation_bytes(w, batch, n_rot):
    """One of n_rot hoisted rotations of a ciphertext: its input once per
    n_rot rotations, one Galois key per batch, the output."""
    n, L, K = 1 << w.log_n, len(w.q_bits), len(w.p_bits)
    alpha = -(-L // w.dnum)
    ndig = -(-L // alpha)
    return 8 * n * (2 * L / n_rot + ndig * 2 * (L + K) / batch + 2 * L)


def bootstrap_bytes(ks_hist, w, batch):
    """The bootstrap's key-switch traffic per ciphertext: sum over its key
    switches at level l of input (2 (l+1) limbs) + key (digits x 2 x (l+1+K)
    limbs, shared by the batch) + output (2 l limbs)."""
    n, K = 1 << w.log_n, len(w.p_bits)
    alpha = -(-len(w.q_bits) // w.dnum)
    words = 0.0
    for lvl, cnt in enumerate(ks_hist):
        if cnt:
            ndig = -(-(lvl + 1) // alpha)
            words += cnt / batch * (2 * (lvl + 1) + ndig * 2 * (lvl + 1 + K) / batch + 2 * lvl)
    return 8 * n * words


def run_gpu(args):
    import torch
    import paper_2506_19693_gb300 as ck

    rank, world, local = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    w = si.PLAIN
    B = 8 if args.small else w.batch
    level = len(w.q_bits) - 1
    scale = 2.0 ** w.log2_scale
    stream = torch.cuda.current_stream()
    ctx = ck.Context.from_workload(w, stream=stream)
    ctx.keygen(1, rot_steps=list(w.rot_steps))
    seed = shard_seeds(rank)
    z = si.messages(seed["mul"], 2 * B, w.slots)
    seeds = si.enc_seeds(seed["mul"], 2 * B)
    cts = [ctx.encrypt(ctx.encode(z[i], level, scale), level, scale, seeds[i]) for i in range(2 * B)]
    A, Bc = cts[:B], cts[B:]
    OUT = [ctx.new_ct(level + 1) for _ in range(B)]
    ROT = [ctx.new_ct(level + 1) for _ in range(B * len(w.rot_steps))]

    # bootstrapping workload: N = 2^16, 2^15 slots, 16 exhausted (level-0) ciphertexts
    wb = si.BOOT
    nb = 2 if args.small else wb.batch
    bctx = ck.Context.from_workload(wb, stream=stream)
    bctx.keygen_boot(2)
    bctx.boot_setup()
    db = 2.0 ** wb.log2_scale
    zb = si.messages(seed["boot"], nb, wb.slots)
    bseeds = si.enc_seeds(seed["boot"], nb)
    BIN = [bctx.encrypt(bctx.encode(zb[i], 0, db), 0, db, bseeds[i]) for i in range(nb)]
    BOUT = [bctx.new_ct(len(wb.q_bits) - 16) for _ in range(nb)]

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    # autotuning, untimed: key inner-product group and NTT row tile per context
    tuning = {"ip_group": ctx.tune(level, B), "ntt_rows": ctx.tune_ntt(16),
              "boot_ip_group": bctx.tune(len(wb.q_bits) - 1, nb), "boot_ntt_rows": bctx.tune_ntt(16)}
    tuning["ntt_cluster"] = ctx.ntt_config()["cluster"]
    tuning["finish_rows"] = ctx.finish_rows()
    tuning["boot_finish_rows"] = bctx.finish_rows()
    tuning["boot_ntt_cluster"] = bctx.ntt_config()["cluster"]

    nvtx = torch.cuda.nvtx

    def step(marks=None):
        # NVTX ranges name the phases (ncu --nvtx-include "timed/hmult/" selects one)
        if marks:
            marks[0].record(stream)
            nvtx.range_push("hmult")
        ctx.mul_relin_batch(A, Bc, OUT, rescale=ck.RESCALE_MERGED)
        if marks:
            nvtx.range_pop()
            marks[1].record(stream)
            nvtx.range_push("rotations")
        ctx.rotate_hoisted(A, list(w.rot_steps), ROT)
        if marks:
            nvtx.range_pop()
            marks[2].record(stream)
            nvtx.range_push("bootstrap")
        bctx.bootstrap_batch(BIN, BOUT)
        if marks:
            nvtx.range_pop()
            marks[3].record(stream)

    def spot_errors():
        got = ctx.decrypt_decode(OUT[0])
        e_mul = float(np.max(np.abs(got - z[0] * z[B])))
        kk = len(w.rot_steps) - 1
        got = ctx.decrypt_decode(ROT[kk * B])
        e_rot = float(np.max(np.abs(got - np.roll(z[0], -w.rot_steps[kk]))))
        e_boot = float(max(np.max(np.abs(bctx.decrypt_decode(BOUT[i]) - zb[i])) for i in range(2)))
        return {"hmult_rescale": e_mul, "rotation": e_rot, "bootstrap": e_boot}

    def timed(form, warmup, clocks=None):
        """Warm-up, spot checks, then `args.steps` timed steps in one form."""
        ctx.set_form(form)
        bctx.set_form(form)
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        errs = spot_errors()
        barrier()
        torch.cuda.synchronize()
        if clocks is not None:
            clocks.start()
        ctx.profile(True)
        bctx.profile(True)
        launches0 = ctx.launch_count() + bctx.launch_count()
        marks = [[ev(), ev(), ev(), ev()] for _ in range(args.steps)]
        torch.cuda.nvtx.range_push("timed")  # ncu --nvtx-include "timed/" selects these launches
        for s in range(args.steps):
            step(marks[s])
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        launches = ctx.launch_count() + bctx.launch_count() - launches0
        hist_p, hist_b = ctx.ks_histogram(), bctx.ks_histogram()
        prof_p, prof_b = ctx.profile_read(), bctx.profile_read()
        parts = [part(prof_p, hist_p, w), part(prof_b, hist_b, wb)]
        prof = dict(prof_p)
        for k, v in prof_b.items():
            a = prof.get(k, (0.0, 0, 0))
            prof[k] = (a[0] + v[0], a[1] + v[1], a[2] + v[2])
        ctx.profile(False)
        bctx.profile(False)
        barrier()
        clk = clocks.stop() if clocks is not None else None
        if ctx.device_error() or bctx.device_error():
            raise RuntimeError(f"device wait expired in the {form} form")
        mul_ms, rot_ms, boot_ms, step_ms = max_over_ranks(
            [sum(m[0].elapsed_time(m[1]) for m in marks), sum(m[1].elapsed_time(m[2]) for m in marks),
             sum(m[2].elapsed_time(m[3]) for m in marks), sum(m[0].elapsed_time(m[3]) for m in marks) / args.steps],
            dist, "cuda")
        return {"mul_ms": mul_ms, "rot_ms": rot_ms, "boot_ms": boot_ms, "step_ms": step_ms, "prof": prof,
                "parts": parts, "launches": launches, "errors": errs, "clocks": clk,
                **job_rates(world, B, len(w.rot_steps), nb, args.steps, mul_ms, rot_ms, boot_ms)}

    main = timed(args.form, args.warmup, ClockSampler(local))
    mul_ms, rot_ms, boot_ms, step_ms = main["mul_ms"], main["rot_ms"], main["boot_ms"], main["step_ms"]
    prof, launches, clk = main["prof"], main["launches"], main["clocks"]
    value, rot_rate, boot_rate = main["hmult_per_s"], main["rotations_per_s"], main["bootstraps_per_s"]
    errors = main["errors"]

    # the same products with ModDown then rescale as two steps (C9, C10)
    e0, e1 = ev(), ev()
    ctx.mul_relin_batch(A, Bc, OUT, rescale=ck.RESCALE_SEPARATE)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        ctx.mul_relin_batch(A, Bc, OUT, rescale=ck.RESCALE_SEPARATE)
    e1.record(stream)
    torch.cuda.synchronize()
    hmult_separate = world * B * args.steps / (max_over_ranks([e0.elapsed_time(e1)], dist, "cuda")[0] / 1e3)

    # roofline of the dominant kernel class
    hbm, tflops, peak_kind = peaks()
    alu = ctx.alu_peaks()
    roof = roofline(main["parts"], hbm, peak_kind, alu, tflops)

    def phase_profiles():
        """One more step, profiled phase by phase: each phase's kernel work and
        key switches by level (for the op-level roofline)."""
        out = {}
        for name, fn, c, wl in (("hmult", lambda: ctx.mul_relin_batch(A, Bc, OUT, rescale=ck.RESCALE_MERGED), ctx, w),
                                ("rotations", lambda: ctx.rotate_hoisted(A, list(w.rot_steps), ROT), ctx, w),
                                ("bootstrap", lambda: bctx.bootstrap_batch(BIN, BOUT), bctx, wb)):
            torch.cuda.synchronize()
            c.profile(True)
            fn()
            torch.cuda.synchronize()
            hist = c.ks_histogram()
            out[name] = (part(c.profile_read(), hist, wl), hist)
            c.profile(False)
        return out

    def op_rooflines(r):
        ph = phase_profiles()
        # the profiled pass is one step: its ops over one step's device time
        hm = op_roofline([ph["hmult"][0]], B, r["mul_ms"] / args.steps / 1e3, hbm, alu, tflops,
                         hmult_bytes(w, B))
        hm["bytes_model"] = ("2 inputs + the relinearisation key / batch + the product one level down "
                             "(the fused minimum)")
        ro = op_roofline([ph["rotations"][0]], B * len(w.rot_steps), r["rot_ms"] / args.steps / 1e3, hbm,
                         alu, tflops, rotation_bytes(w, B, len(w.rot_steps)))
        ro["bytes_model"] = "the input once per 15 hoisted rotations + one Galois key / batch + the output"
        bo = op_roofline([ph["bootstrap"][0]], nb, r["boot_ms"] / args.steps / 1e3, hbm, alu, tflops,
                         bootstrap_bytes(ph["bootstrap"][1], wb, nb))
        bo["bytes_model"] = ("sum over the circuit's key switches at level l of input (2(l+1) limbs) + key "
                             "(digits x 2(l+1+K) limbs) / batch + output (2l limbs)")
        bo["key_switches_per_bootstrap"] = sum(ph["bootstrap"][1]) / nb
        bo["key_switches_by_level"] = {lvl: c / nb for lvl, c in enumerate(ph["bootstrap"][1]) if c}
        return {"hmult": hm, "rotation": ro, "bootstrap": bo}

    op_roofs = op_rooflines(main)

    # the same three phases in the other basis-conversion form, for comparison
    forms = {}
    if not args.no_form_compare:
        runs = [(args.form, main, op_roofs)]
        for other in FORM_NAMES:
            if other != args.form:
                r = timed(other, 2)
                runs.append((other, r, op_rooflines(r)))
        ctx.set_form(args.form)
        bctx.set_form(args.form)
        for f, r, orf in runs:
            conv = {"tensor": "bconv_tc", "uint64": "bconv", "fused": "conv_fused"}[f]
            total = sum(timed_classes(r["parts"]).values())
            forms[f] = {"hmult_per_s": r["hmult_per_s"], "rotations_per_s": r["rotations_per_s"],
                        "bootstraps_per_s": r["bootstraps_per_s"], "slot_error": r["errors"],
                        "basis_conversion_share": timed_classes(r["parts"]).get(conv, 0.0) / total,
                        "basis_conversion_roofline": roofline(r["parts"], hbm, peak_kind, alu, tflops, name=conv),
                        "dominant_kernel_roofline": roofline(r["parts"], hbm, peak_kind, alu, tflops),
                        "op_rooflines": {k: {"frac": v["frac"], "bound": v["bound"], "hbm_frac": v["hbm"]["frac"],
                                             "compute_frac": v["compute"]["frac"]} for k, v in orf.items()}}

    # ReBoot RE-Block training step (Alg. 1 + Alg. 2 + Bootstrap of W, V), the
    # synthetic MLP workload: 128 samples x 784 features in [0, 1], 784 -> 128 -> 10,
    # r x c = 256 x 128, on the bootstrapping context
    reboot = None
    if not (args.no_reboot or args.small):
        reboot = run_reboot_step(bctx, wb, torch, stream, rank)
    n_scaling = None
    if not (args.no_n_scaling or args.small):
        n_scaling = run_n_scaling(torch, stream, reps=max(2, min(args.steps, 3)))
    key_compression = None
    if not (args.no_key_compression or args.small):
        key_compression = run_key_compression(torch, stream, max(3, min(args.steps, 5)), args.form)
    sparse_boot = None
    if not (args.no_sparse_boot or args.small):
        sparse_boot = run_sparse_boot(torch, stream, max(2, min(args.steps, 3)), args.form)
    iterative = None
    if not (args.no_iterative or args.small):
        iterative = run_iterative(bctx, wb, BIN, BOUT, zb, torch, stream, reps=max(2, min(args.steps, 3)))
    uneven = None
    if not (args.no_uneven or args.small):
        uneven = run_uneven(ctx, w, torch, stream, rank, reps=max(3, args.steps), warmup=args.warmup,
                            hbm_peak=hbm)
        ctx.set_form(args.form)

    tc_ntt = None
    if not (args.no_tc_ntt or args.small):
        tc_ntt = run_tc_ntt_prototype(ctx, w, torch, stream, reps=max(2, min(args.steps, 3)))
    cluster_ntt = None
    if not (args.no_tc_ntt or args.small):
        cluster_ntt = run_cluster_ntt(ctx, w, torch, stream, max(2, min(args.steps, 3)), A, Bc, OUT)
    finish = None
    if not (args.no_finish_compare or args.small):
        finish = run_fused_finish(ctx, bctx, w, torch, stream, max(2, min(args.steps, 3)), A, Bc, OUT, ROT, BIN,
                                  BOUT)
    tc_inner = None
    if not (args.no_tc_ntt or args.small):
        tc_inner = run_tc_inner_prototype(torch, stream, max(2, min(args.steps, 3)))

    # end-to-end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not (args.no_e2e or args.small):
        e2e = run_e2e(ctx, torch, A, Bc, OUT, level, args, dist)

    # the gadget size for this prime chain (informational; the workload keeps dnum = 3)
    if not args.small:
        best_d, ms_d = ck.tune_dnum(w, cands=(2, 3, 4, 6), batch=8)
        tuning["dnum_best"] = best_d
        tuning["dnum_ms_per_hmult"] = {d: (round(v, 4) if v != float("inf") else None) for d, v in ms_d.items()}

    cpu = None
    if rank == 0 and world == 1 and not (args.no_cpu_baseline or args.small):
        sample = OracleSample(w)
        dt, threads = sample.time(), sample.threads
        dr = sample.time_rotation(1)
        cpu = {"value": 1.0 / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "1 HMult+relin+rescale of 1 ciphertext pair at N=2^16, L=24 (1/64 of the batch)",
               "rotations_per_s": 1.0 / dr,
               "rotation_sample": "1 rotation by 1 slot of 1 ciphertext at N=2^16, L=24 (key generated untimed)"}

    # the metric's op-level fractions and the other half of the metric (bootstraps/s),
    # per form, as flat scalars of the roofline object
    if roof is not None:
        for k, v in op_roofs.items():
            roof[f"op_{k}_per_s"] = v["ops_per_s"]
            roof[f"op_{k}_frac"] = v["frac"]
            roof[f"op_{k}_bound"] = v["bound"]
            roof[f"op_{k}_hbm_frac"] = v["hbm"]["frac"]
            roof[f"op_{k}_compute_frac"] = v["compute"]["frac"]
        roof["bootstraps_per_s"] = boot_rate
        for f, r in forms.items():
            roof[f"form_{f}_hmult_per_s"] = r["hmult_per_s"]
            roof[f"form_{f}_bootstraps_per_s"] = r["bootstraps_per_s"]
            roof[f"form_{f}_rotations_per_s"] = r["rotations_per_s"]

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": config_of(w, B, args.form),
                "rotations_per_s": rot_rate, "bootstraps_per_s": boot_rate,
                "hmult_separate_rescale_per_s": hmult_separate,
                "phase_ms_per_step": {"hmult_relin_rescale_x64": mul_ms / args.steps,
                                      "rotations_hoisted_64x15": rot_ms / args.steps,
                                      "bootstrap_x16": boot_ms / args.steps},
                "bootstrap_config": {"workload": wb.name, "log_n": wb.log_n, "slots": wb.slots,
                                     "n_q": len(wb.q_bits), "n_p": len(wb.p_bits), "dnum": wb.dnum,
                                     "batch": nb, "levels_consumed": 16, "cheb_degree": 60,
                                     "double_angles": 3, "input": "fresh encryptions at level 0"},
                "slot_error": errors, "forms": forms,
                "reboot_step": reboot, "uneven_batch": uneven, "iterative_bootstrap": iterative,
                "n_scaling": n_scaling,
                "key_compression": key_compression,
                "sparse_slot_bootstrap": sparse_boot,
                "tensor_ntt_stage_prototype": tc_ntt,
                "cluster_ntt": cluster_ntt,
                "fused_finish": finish,
                "tensor_inner_product_prototype": tc_inner,
                "tuning": tuning,
                "e2e": e2e, "roofline": roof, "op_rooflines": op_roofs, "alu_peaks": alu, "cpu_baseline": cpu,
                "clocks": clk,
                "gpu_launches": int(launches),
                "kernel_ms": {k: round(v[0], 3) for k, v in prof.items() if v[1]},
                "kernel_rooflines": kernel_rooflines(main["parts"], hbm, peak_kind, alu, tflops)}
        print(json.dumps(line))
    bctx.close()
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_uneven(ctx16, w, torch, stream, rank, reps, warmup, dnums=(3, 2), hbm_peak=None):
    """256 independent operations over ring degrees 2^15 / 2^16 (p = 1/2) with
    limb counts uniform in 4..24 (level index 3..23), one third each
    HMult+relin(+rescale), rotation by a random power of two and rescale;
    captured as one CUDA graph and replayed, in both basis-conversion forms and
    for each gadget in `dnums` (3: the workload's; 2: the tuner's choice for
    this chain), the same inputs every time.  Returns ops/s of the replays, of
    the eager first run, and the algorithmic bytes of one replay."""
    import paper_2506_19693_gb300 as ck
    ctxs = {}  # (dnum, log_n) -> context
    for d in dnums:
        alpha = -(-len(w.q_bits) // d)
        for log_n in (15, 16):
            if d == w.dnum and log_n == 16:
                c = ctx16
            else:
                c = ck.Context(log_n, w.q_bits, (w.p_bits[0],) * alpha, d, w.h, w.sigma, w.log2_scale, stream=stream)
                c.keygen(5 if log_n == 15 else 1, rot_steps=[1 << k for k in range(log_n - 2)])
                c._owned_by_uneven = True
            ctxs[(d, log_n)] = c
    tuned = {}
    for (d, log_n), c in ctxs.items():
        tuned[f"dnum{d}_n{1 << log_n}"] = {"ip_group": c.tune(len(w.q_bits) - 1, 64), "ntt_rows": c.tune_ntt(16)}
    rng = np.random.default_rng(shard_seeds(rank)["uneven"])
    scale = 2.0 ** w.log2_scale
    specs = []  # (log_n, kind, a, b, out, k)
    n_bytes = 0.0
    keys = set()
    for i in range(256):
        log_n = 16 if rng.random() < 0.5 else 15
        c = ctxs[(w.dnum, log_n)]
        level = int(rng.integers(3, len(w.q_bits)))  # 4..24 limbs
        z = si.messages(600 + i, 2, c.n // 2)
        a = c.encrypt(c.encode(z[0], level, scale), level, scale, 900000 + i)
        out = c.new_ct(level + 1)
        kind = i % 3
        limb = 8 * c.n
        b, k = None, 0
        if kind == 0:
            b = c.encrypt(c.encode(z[1], level, scale), level, scale, 950000 + i)
            n_bytes += limb * (2 * 2 * (level + 1) + 2 * level)
            keys.add((log_n, 0, level))
        elif kind == 1:
            k = int(1 << rng.integers(0, c.log_n - 2))
            n_bytes += limb * 2 * 2 * (level + 1)
            keys.add((log_n, k, level))
        else:
            n_bytes += limb * (2 * (level + 1) + 2 * level)
        specs.append((log_n, kind, a, b, out, k))
    alpha = -(-len(w.q_bits) // w.dnum)
    for log_n, _, level in keys:  # each key group reads its key once per replay (dnum 3)
        n_bytes += 8 * (1 << log_n) * (-(-(level + 1) // alpha)) * 2 * (level + 1 + len(w.p_bits))

    def ops_for(d):
        ops = []
        for log_n, kind, a, b, out, k in specs:
            c = ctxs[(d, log_n)]
            if kind == 0:
                ops.append(ck.Op(c, ck.OP_MUL_RELIN, a, out, b=b, rescale=True))
            elif kind == 1:
                ops.append(ck.Op(c, ck.OP_ROTATE, a, out, k=k))
            else:
                ops.append(ck.Op(c, ck.OP_RESCALE, a, out))
        return ops

    torch.cuda.synchronize()
    gs = torch.cuda.Stream()  # captured graphs replay on a created stream; time on that stream
    res = {}
    eager = None
    try:
        for d in dnums:
            for form in ("uint64", "tensor", "fused"):
                for (dd, _), c in ctxs.items():
                    if dd == d:
                        c.set_form(form)
                ops = ops_for(d)
                if eager is None:
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    ck.execute(ops)
                    torch.cuda.synchronize()
                    eager = time.perf_counter() - t0
                g = ck.Graph(ops, stream=gs)
                for _ in range(warmup):
                    g.launch()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(gs)
                for _ in range(reps):
                    g.launch()
                e1.record(gs)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                g.close()
                row = {"ops_per_s_graph": 256 / (ms / 1e3), "ms_per_batch_graph": ms}
                if d == w.dnum and hbm_peak:
                    row["hbm_frac"] = n_bytes / (ms / 1e3) / (hbm_peak * 1e9)
                res[f"dnum{d}_{form}"] = row
    finally:
        for c in ctxs.values():
            c.set_form(False)
        for c in ctxs.values():
            if getattr(c, "_owned_by_uneven", False):
                c.close()
    best = max(res, key=lambda k: res[k]["ops_per_s_graph"])
    return {"forms": res, "best": best, "ops_per_s_graph": res[best]["ops_per_s_graph"],
            "ops_per_s_eager_first_run": 256 / eager,
            "algorithmic_bytes_per_batch": n_bytes,
            "bytes_model": "per op its inputs and output at their levels, plus each (ring, key, level) group's "
                           "switching key once (dnum 3)",
            "ops": "256: 1/3 HMult+relin+rescale, 1/3 Rot(2^k), 1/3 rescale; N in {2^15, 2^16} p=1/2; "
                   "limbs U{4..24} (level index 3..23)", "replays": reps, "tuned": tuned}


def run_tc_ntt_prototype(ctx, w, torch, stream, reps, n_polys=64):
    """The tensor-core NTT stage group (ckks_ntt_tc: the first four column
    stages as a byte-split tcgen05 GEMM) against the uint64 transform on the
    same 64 polynomials x 24 limbs; the profiler splits the prototype's time
    into the tensor-core stage group and the CUDA-core stages after it."""
    import paper_2506_19693_gb300 as ck
    L = len(w.q_bits)
    n = ctx.n
    g = torch.Generator(device=ctx.device)
    g.manual_seed(5)
    data = torch.empty((n_polys, L, n), dtype=torch.int64, device=ctx.device)
    for t in range(L):
        data[:, t] = torch.randint(0, int(ctx.q[t]), (n_polys, n), device=ctx.device, generator=g)
    a = data.clone()
    b = data.clone()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    ctx.ntt_tc(a, n_polys, L)  # warm-up (builds the byte-plane matrices)
    for p in range(n_polys):
        ctx.ntt(b[p], 0)
    torch.cuda.synchronize()
    same = bool(torch.equal(a, b))
    e0, e1, e2 = ev(), ev(), ev()
    e0.record(stream)
    for _ in range(reps):
        ctx.ntt_tc(a, n_polys, L)
    e1.record(stream)
    for _ in range(reps):
        for p in range(n_polys):
            ctx.ntt(b[p], 0)
    e2.record(stream)
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.ntt_tc(a, n_polys, L)
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    stage_ms = prof.get("bconv_tc", (0.0, 0, 0))[0]
    rest_ms = prof.get("ntt_fwd_pass_a", (0.0, 0, 0))[0] + prof.get("ntt_fwd_pass_b", (0.0, 0, 0))[0]
    limbs = n_polys * L
    # the stage group: a 16 x 16 product per 16-point block = 16 MACs per value,
    # as byte-split fp16 MMAs: 8 x 8 byte products each, 2 flops each
    tc_flops = limbs * n * 16 * 64 * 2
    return {"limbs": limbs, "bit_exact_vs_uint64": same,
            "ms_tensor_stage_ntt": e0.elapsed_time(e1) / reps, "ms_uint64_ntt": e1.elapsed_time(e2) / reps,
            "stage_group_ms": stage_ms, "remaining_stages_ms": rest_ms,
            "stage_group_us_per_limb": 1e3 * stage_ms / limbs,
            "stage_group_tensor_tflops": tc_flops / (stage_ms / 1e3) / 1e12 if stage_ms else None,
            "note": "uint64 NTT launched per polynomial (24 limbs per launch); the four stages the prototype moves "
                    "to the tensor cores are half of the uint64 column pass"}


def run_tc_inner_prototype(torch, stream, reps):
    """The key-switch inner product of 128 ciphertexts sharing one key (3
    digits, all 32 limbs of the N = 2^16 chain) as a byte-split tcgen05 GEMM
    (ckks_ks_inner_tc) against the same product on the CUDA cores
    (ckks_ks_inner_u64), on identical random residues."""
    import paper_2506_19693_gb300 as ck
    w = si.PLAIN
    ctx = ck.Context.from_workload(w, stream=stream)
    P, ndig = 128, 3
    L, n = len(ctx.moduli), ctx.n
    g = torch.Generator(device=ctx.device)
    g.manual_seed(9)
    d = torch.empty((P, ndig, L, n), dtype=torch.int64, device=ctx.device)
    key = torch.empty((ndig, 2, L, n), dtype=torch.int64, device=ctx.device)
    for t in range(L):
        q = int(ctx.moduli[t])
        d[:, :, t] = torch.randint(0, q, (P, ndig, n), device=ctx.device, generator=g)
        key[:, :, t] = torch.randint(0, q, (ndig, 2, n), device=ctx.device, generator=g)
    outs = {f: torch.empty((P, 2, L, n), dtype=torch.int64, device=ctx.device) for f in ("tensor", "uint64")}
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    ms = {}
    for f in ("tensor", "uint64"):
        ctx.ks_inner(d, key, outs[f], f)
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        for _ in range(reps):
            ctx.ks_inner(d, key, outs[f], f)
        e1.record(stream)
        torch.cuda.synchronize()
        ms[f] = e0.elapsed_time(e1) / reps
    same = bool(torch.equal(outs["tensor"], outs["uint64"]))
    err = ctx.device_error()
    ctx.close()
    pairs = P * L * n  # output pairs (o = 0, 1)
    flops = pairs * 16 * (8 * ndig) * 2  # one 16-column row of the byte GEMM per output pair
    hbm_bytes = 8 * L * n * (P * ndig + 2 * ndig + 2 * P)
    return {"ciphertexts": P, "digits": ndig, "limbs": L, "bit_exact_vs_uint64": same, "device_error": err,
            "ms_tensor": ms["tensor"], "ms_uint64": ms["uint64"],
            "tensor_tflops": flops / (ms["tensor"] / 1e3) / 1e12,
            "hbm_gbs_tensor": hbm_bytes / (ms["tensor"] / 1e3) / 1e9,
            "hbm_gbs_uint64": hbm_bytes / (ms["uint64"] / 1e3) / 1e9,
            "note": "bytes: the digits, the key and the outputs once each"}


def run_fused_finish(ctx, bctx, w, torch, stream, reps, A, Bc, OUT, ROT, BIN, BOUT):
    """The key-switch finish in the forward NTT's row pass (both row tiles)
    against a separate kernel after the transform: the three phases of the step
    timed with each (CUDA events), and the outputs compared bit for bit."""
    import paper_2506_19693_gb300 as ck
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    phases = [("hmult_ms", lambda: ctx.mul_relin_batch(A, Bc, OUT, rescale=ck.RESCALE_MERGED), reps),
              ("rotations_ms", lambda: ctx.rotate_hoisted(A, list(w.rot_steps), ROT), reps),
              ("bootstrap_ms", lambda: bctx.bootstrap_batch(BIN, BOUT), max(1, reps - 1))]
    res, outs = {}, {}
    tuned = (ctx.finish_rows(), bctx.finish_rows())
    for on, rows in ((False, 0), (True, 16), (True, 8)):
        ctx.set_fused_finish(on)
        bctx.set_fused_finish(on)
        if on:
            ctx.set_finish_rows(rows)
            bctx.set_finish_rows(rows)
        r = {}
        for key, fn, k in phases:
            fn()
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record(stream)
            for _ in range(k):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            r[key] = e0.elapsed_time(e1) / k
        res[f"fused_rows{rows}" if on else "separate"] = r
        outs[rows] = [ctx.export_ct(OUT[0]), ctx.export_ct(ROT[-1]), bctx.export_ct(BOUT[0])]
    ctx.set_finish_rows(tuned[0])
    bctx.set_finish_rows(tuned[1])
    res["tuned_rows"] = {"main": tuned[0], "bootstrap": tuned[1]}
    res["bit_exact"] = all(bool(np.array_equal(x, y)) for r in (16, 8) for x, y in zip(outs[0], outs[r]))
    return res


def run_cluster_ntt(ctx, w, torch, stream, reps, A, Bc, OUT):
    """The forward NTT in one pass on 8-CTA clusters (each limb read and written
    once) against the two passes (each limb crosses HBM twice), on the bench's
    merged HMult batch: batch time and the profiler's forward-transform time per
    limb in each form.  Both forms give identical limbs (checked here too)."""
    import paper_2506_19693_gb300 as ck
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    was = ctx.ntt_config()["cluster"]
    # like for like: the fused key-switch finish always takes the two passes
    ctx.set_fused_finish(False)
    res = {}
    outs = {}
    for on in (False, True):
        res_key = "cluster" if on else "two_pass"
        info = ctx.set_ntt_cluster(on)
        ctx.mul_relin_batch(A, Bc, OUT, rescale=ck.RESCALE_MERGED)
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        for _ in range(reps):
            ctx.mul_relin_batch(A, Bc, OUT, rescale=ck.RESCALE_MERGED)
        e1.record(stream)
        torch.cuda.synchronize()
        ctx.profile(True)
        ctx.profile_read()
        ctx.mul_relin_batch(A, Bc, OUT, rescale=ck.RESCALE_MERGED)
        torch.cuda.synchronize()
        prof = ctx.profile_read()
        ctx.profile(False)
        outs[on] = ctx.export_ct(OUT[0])
        kinds = ("ntt_fwd_cluster",) if on else ("ntt_fwd_pass_a", "ntt_fwd_pass_b")
        fwd_ms = sum(prof.get(k, (0.0, 0, 0))[0] for k in kinds)
        limbs = prof.get(kinds[0], (0.0, 0, 0))[2]
        res[res_key] = {"ms_per_batch": e0.elapsed_time(e1) / reps, "forward_ntt_ms": fwd_ms,
                        "forward_limbs": limbs, "us_per_limb": 1e3 * fwd_ms / limbs if limbs else None,
                        "hbm_bytes_per_limb": (1 if on else 2) * 2 * 8 * ctx.n}
        if on:
            res[res_key]["resident_clusters"] = info
    ctx.set_ntt_cluster(was)
    ctx.set_fused_finish(True)
    res["bit_exact"] = bool(np.array_equal(outs[False], outs[True]))
    res["note"] = "key-switch finish in a separate kernel for both forms"
    return res


def run_n_scaling(torch, stream, reps):
    """Ring-degree scaling (the paper's Fig. 3 axis): merged HMult+relin+rescale
    on the 24 + 8 prime chain at N = 2^15, 2^16, 2^17 with the same number of
    coefficients per batch (128, 64, 32 pairs), and bootstrapping at N = 2^17
    (2^16 slots, Table 3's eMLP-2 chain l = 27, 8 ciphertexts)."""
    import paper_2506_19693_gb300 as ck
    w = si.PLAIN
    level = len(w.q_bits) - 1
    scale = 2.0 ** w.log2_scale
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    out = {"hmult": {}}
    for log_n in (15, 16, 17):
        ctx = ck.Context(log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma, w.log2_scale, stream=stream)
        try:
            ctx.keygen(9)
            B = 64 << 16 >> log_n
            z = si.messages(700 + log_n, 2, 1 << (log_n - 1))
            base = [ctx.encrypt(ctx.encode(z[i], level, scale), level, scale, 900 + i) for i in range(2)]
            cts = [ctx.new_ct(level + 1) for _ in range(2 * B)]
            for i, c in enumerate(cts):  # pairs (base 0, base 1)
                c.data.copy_(base[i // B].data)
                c.level, c.scale = base[i // B].level, base[i // B].scale
            outs = [ctx.new_ct(level + 1) for _ in range(B)]
            ctx.tune(level, B)
            ctx.tune_ntt(16)
            ctx.mul_relin_batch(cts[:B], cts[B:], outs, rescale=ck.RESCALE_MERGED)
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record(stream)
            for _ in range(reps):
                ctx.mul_relin_batch(cts[:B], cts[B:], outs, rescale=ck.RESCALE_MERGED)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            err = float(np.max(np.abs(ctx.decrypt_decode(outs[0]) - z[0] * z[1])))
            out["hmult"][f"n{1 << log_n}"] = {"pairs": B, "hmult_per_s": B / (ms / 1e3),
                                              "coeff_hmult_per_s": B * (1 << log_n) / (ms / 1e3),
                                              "ms_per_batch": ms, "slot_error": err}
        finally:
            ctx.close()
    wb = si.BOOT17
    bctx = ck.Context.from_workload(wb, stream=stream)
    try:
        bctx.keygen_boot(2)
        bctx.boot_setup()
        nb = wb.batch
        db = 2.0 ** wb.log2_scale
        zb = si.messages(710, nb, wb.slots)
        seeds = si.enc_seeds(710, nb)
        bin_ = [bctx.encrypt(bctx.encode(zb[i], 0, db), 0, db, seeds[i]) for i in range(nb)]
        bout = [bctx.new_ct(len(wb.q_bits) - 16) for _ in range(nb)]
        bctx.tune(len(wb.q_bits) - 1, nb)
        bctx.tune_ntt(16)
        bctx.bootstrap_batch(bin_, bout)
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        for _ in range(reps):
            bctx.bootstrap_batch(bin_, bout)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        err = float(max(np.max(np.abs(bctx.decrypt_decode(bout[i]) - zb[i])) for i in range(2)))
        out["bootstrap_n131072"] = {"workload": wb.name, "batch": nb, "bootstraps_per_s": nb / (ms / 1e3),
                                    "ms_per_batch": ms, "slot_error": err, "output_level": bout[0].level}
        out["emlp2_step"] = run_emlp_step(bctx, wb, torch, stream, [(784, 64), (64, 32)],
                                          {"eMLP-2 (Table 6, 2x Xeon Gold 5318S)": 629.65})
    finally:
        bctx.close()
    wb3 = si.BOOT17_L29
    bctx = ck.Context.from_workload(wb3, stream=stream)
    try:
        bctx.keygen_boot(3)
        bctx.boot_setup()
        bctx.tune(len(wb3.q_bits) - 1, 8)
        bctx.tune_ntt(16)
        out["emlp3_step"] = run_emlp_step(bctx, wb3, torch, stream, [(784, 128), (128, 64), (64, 32)],
                                          {"eMLP-3": "not in Table 6"})
    finally:
        bctx.close()
    out["clock"] = "CUDA events on the library stream, inputs resident; untimed tuning and warm-up"
    return out


def run_sparse_boot(torch, stream, reps, form, log_slots=13):
    """Sparse-slot bootstrapping at N = 2^16 (reading B13): 2^13-slot messages
    repeated 4 times across the 2^15 slots, 16 ciphertexts per batch on the
    bootstrapping chain (25 + 9 primes), fresh encryptions at level 0."""
    import paper_2506_19693_gb300 as ck
    wb = si.BOOT
    ctx = ck.Context.from_workload(wb, stream=stream)
    try:
        ctx.set_form(form)
        ctx.boot_set_slots(1 << log_slots)
        ctx.keygen_boot(4)
        ctx.boot_setup()
        nb = wb.batch
        db = 2.0 ** wb.log2_scale
        reps_copies = wb.slots >> log_slots
        zb = si.messages(730, nb, 1 << log_slots)
        seeds = si.enc_seeds(730, nb)
        bin_ = [ctx.encrypt(ctx.encode(np.tile(zb[i], reps_copies), 0, db), 0, db, seeds[i]) for i in range(nb)]
        bout = [ctx.new_ct(len(wb.q_bits) - 16) for _ in range(nb)]
        ctx.tune(len(wb.q_bits) - 1, nb)
        ctx.tune_ntt(16)
        ctx.bootstrap_batch(bin_, bout)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ctx.bootstrap_batch(bin_, bout)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        err = float(max(np.max(np.abs(ctx.decrypt_decode(bout[i]) - np.tile(zb[i], reps_copies)))
                        for i in range(2)))
        return {"workload": wb.name, "slots": 1 << log_slots, "batch": nb, "bootstraps_per_s": nb / (ms / 1e3),
                "ms_per_batch": ms, "slot_error": err, "output_level": bout[0].level,
                "clock": "CUDA events on the library stream, inputs resident; untimed tuning and warm-up"}
    finally:
        ctx.close()


def run_key_compression(torch, stream, reps, form):
    """Compressed switching keys (b rows plus the generator state of a) against
    full keys, on the HMult workload: merged HMult+relin+rescale over 64 pairs and
    over 1 pair, and one input rotated by the 15 powers of two in one hoisted
    call.  Results are bit-identical; what changes is key memory and key reads."""
    import paper_2506_19693_gb300 as ck
    w = si.PLAIN
    level = len(w.q_bits) - 1
    scale = 2.0 ** w.log2_scale
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    out = {}
    for compressed in (False, True):
        ctx = ck.Context.from_workload(w, stream=stream)
        try:
            ctx.set_key_compression(compressed)
            ctx.set_form(form)
            ctx.keygen(9, rot_steps=list(w.rot_steps))
            z = si.messages(720, 2, w.slots)
            base = [ctx.encrypt(ctx.encode(z[i], level, scale), level, scale, 920 + i) for i in range(2)]
            B = w.batch
            cts = [ctx.new_ct(level + 1) for _ in range(2 * B)]
            for i, c in enumerate(cts):
                c.data.copy_(base[i // B].data)
                c.level, c.scale = base[i // B].level, base[i // B].scale
            outs = [ctx.new_ct(level + 1) for _ in range(B)]
            rots = [ctx.new_ct(level + 1) for _ in w.rot_steps]
            ctx.tune(level, B)
            ctx.tune_ntt(16)

            def time_it(fn, n):
                fn()
                torch.cuda.synchronize()
                e0, e1 = ev(), ev()
                e0.record(stream)
                for _ in range(n):
                    fn()
                e1.record(stream)
                torch.cuda.synchronize()
                return e0.elapsed_time(e1) / n

            ms64 = time_it(lambda: ctx.mul_relin_batch(cts[:B], cts[B:], outs, rescale=ck.RESCALE_MERGED), reps)
            ms1 = time_it(lambda: ctx.mul_relin_batch(cts[:1], cts[B:B + 1], outs[:1],
                                                      rescale=ck.RESCALE_MERGED), 16 * reps)
            msr = time_it(lambda: ctx.rotate_hoisted(cts[:1], list(w.rot_steps), rots), 4 * reps)
            n_keys = 1 + len(w.rot_steps)
            words = ctx.n_digits * (ctx.n_q + ctx.n_p) * ctx.n * (1 if compressed else 2) + (16 if compressed else 0)
            row = {"device_key_mb": n_keys * words * 8 / 1e6,
                   "hmult_per_s_64_pairs": B / (ms64 / 1e3), "hmult_ms_1_pair": ms1,
                   "hoisted_15_rotations_ms_1_input": msr,
                   "slot_error": float(np.max(np.abs(ctx.decrypt_decode(outs[0]) - z[0] * z[1])))}
            out["compressed" if compressed else "full"] = row
        finally:
            ctx.close()
    out["clock"] = "CUDA events on the library stream, inputs resident; untimed tuning and warm-up"
    return out


def run_emlp_step(bctx, wb, torch, stream, dims, paper_s, b=128):
    """One training step of an eMLP of Table 3 at N = 2^17 (r = c = 256): blocks
    alternate RE, CE, RE (reading R6 for the CE-Block), each block fed the
    previous block's activations and bootstrapping its weights and
    velocities.  b synthetic samples; one untimed warm-up iteration, one timed
    iteration (NAG with velocity)."""
    import paper_2506_19693_gb300.reboot as rb
    gs = [rb.Geometry(256, 256, k0, k1, 10) for k0, k1 in dims]
    for k in sorted(set(gs[0].rotation_steps())):
        bctx.keygen_galois(bctx.galois_elt(k))
    rng = np.random.default_rng(800 + len(dims))
    x = rng.uniform(0, 1, size=(b, dims[0][0]))
    y = np.eye(10)[rng.integers(0, 10, size=b)]
    scale, lvl = 2.0 ** wb.log2_scale, len(wb.q_bits) - 17
    seeds = iter(range(3 * 10 ** 6, 4 * 10 ** 6))
    enc = lambda v: bctx.encrypt(bctx.encode(v, lvl, scale), lvl, scale, next(seeds))  # noqa: E731
    zero = np.zeros(256 * 256)
    states, blocks = [], []
    for h, (g, (k0, k1)) in enumerate(zip(gs, dims)):
        w = rng.normal(0, 1 / np.sqrt(k0), size=(k0, k1))
        ws = rng.normal(0, 1 / np.sqrt(k1), size=(k1, 10))
        if h % 2 == 0:  # RE-Block: row-wise tiles, column-wise classifier
            tiles = rb.weight_tiles(w, g)
            states.append(([enc(t) for t in tiles], [enc(zero) for _ in tiles], enc(rb.pack_colwise(ws, g)),
                           enc(zero), None))
            blocks.append(rb.REBlock(bctx, g, 0.001 / b, 0.001, 0.9))
        else:           # CE-Block: column-wise layer, row-wise classifier
            states.append((enc(rb.pack_colwise(w, g)), enc(zero), enc(rb.pack_rowwise(ws, g)), enc(zero), None))
            blocks.append(rb.CEBlock(bctx, g, 0.001 / b, 0.001, 0.9))
    xs = [[enc(t) for t in rb.input_tiles(xi, gs[0])] for xi in x]
    ys_exp = [enc(rb.pack_expanded(yi, gs[0])) for yi in y]
    ys_rep = [enc(rb.pack_repeated(yi, gs[0])) for yi in y]

    def iteration(states, first):
        out, inp = [], xs
        for h, (blk, st) in enumerate(zip(blocks, states)):
            if h % 2 == 0:
                out.append(blk.step(st, inp, ys_exp, first))
            else:
                out.append(blk.step(st, inp, ys_rep, first))
            acts = blk.last_activations
            inp = acts if h % 2 == 0 else [[a] for a in acts]
        return out

    states = iteration(states, True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = bctx.launch_count()
    e0.record(stream)
    states = iteration(states, False)
    e1.record(stream)
    torch.cuda.synchronize()
    nboot = sum(2 * g.tiles + 2 if h % 2 == 0 else 4 for h, g in enumerate(gs))
    return {"seconds_per_step": e0.elapsed_time(e1) / 1e3, "samples": b, "workload": wb.name,
            "blocks": " -> ".join(("RE" if h % 2 == 0 else "CE") + f"({k1})" for h, (_, k1) in enumerate(dims)),
            "geometry": "r = c = 256, 784 inputs in 4 row tiles, classifiers to 10 outputs",
            "bootstraps": nboot, "kernel_launches": bctx.launch_count() - l0,
            "paper_cpu_context_s": paper_s}


def run_iterative(bctx, wb, BIN, BOUT, zb, torch, stream, reps, log2_k=16):
    """The same 16 exhausted ciphertexts through two-pass (iterative)
    bootstrapping (reading B12): throughput and slot error against one pass."""
    bctx.bootstrap_iterative_batch(BIN, log2_k, out=BOUT)  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        bctx.bootstrap_iterative_batch(BIN, log2_k, out=BOUT)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    err = float(max(np.max(np.abs(bctx.decrypt_decode(BOUT[i]) - zb[i])) for i in range(2)))
    return {"bootstraps_per_s": len(BIN) / (ms / 1e3), "ms_per_batch": ms, "batch": len(BIN), "log2_k": log2_k,
            "slot_error": err, "reps": reps, "output_level": BOUT[0].level,
            "clock": "CUDA events on the library stream, inputs resident"}


def run_reboot_step(bctx, wb, torch, stream, rank):
    """One warm-up and one timed RE-Block step at the config-3 size."""
    import paper_2506_19693_gb300.reboot as rb
    g = rb.Geometry(256, 128, 784, 128, 10)
    for k in g.rotation_steps():
        bctx.keygen_galois(bctx.galois_elt(k))
    b = 128
    rng = np.random.default_rng(shard_seeds(rank)["reboot"])
    x = rng.uniform(0, 1, size=(b, g.k0))
    y = np.eye(g.o)[rng.integers(0, g.o, size=b)]
    w = rng.normal(0, 1 / np.sqrt(g.k0), size=(g.k0, g.k1))
    ws = rng.normal(0, 1 / np.sqrt(g.k1), size=(g.k1, g.o))
    scale, lvl = 2.0 ** wb.log2_scale, len(wb.q_bits) - 17
    seeds = iter(range(10 ** 6, 2 * 10 ** 6))
    enc = lambda v: bctx.encrypt(bctx.encode(v, lvl, scale), lvl, scale, next(seeds))  # noqa: E731
    state = ([enc(t) for t in rb.weight_tiles(w, g)], [enc(np.zeros(g.r * g.c)) for _ in range(g.tiles)],
             enc(rb.pack_colwise(ws, g)), enc(np.zeros(g.r * g.c)), None)
    xs = [[enc(t) for t in rb.input_tiles(xi, g)] for xi in x]
    ys = [enc(rb.pack_expanded(yi, g)) for yi in y]
    # gamma 0.001 and eta 0.001, mu 0.9 (MNIST / eMLP-1 hyperparameters), 1/b folded into gamma
    blk = rb.REBlock(bctx, g, 0.001 / b, 0.001, 0.9)
    state = blk.step(state, xs, ys, first=True)  # warm-up (iteration 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = bctx.launch_count()
    e0.record(stream)
    state = blk.step(state, xs, ys, first=False)  # iteration 2: NAG with velocity
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"seconds_per_step": ms / 1e3, "samples": b, "geometry": "r=256 c=128, 784->128->10, 4 input tiles",
            "ops": "per sample 12 ct-ct mult + 30 rotations; NAG on 5 weight cts; 10 bootstraps",
            "kernel_launches": bctx.launch_count() - l0,
            "paper_cpu_context_s": {"eMLP-1 (Table 6, 2x Xeon Gold 5318S)": 190.32}}


def run_e2e(ctx, torch, A, Bc, OUT, level, args, dist):
    """HMult+relin+rescale of the batch from page-locked host memory to
    page-locked host memory through the public host-streamed calls: the copies
    of one chunk overlap the products of the next; all copies inside the timed
    region.  Two wire formats: plain uint64 limbs (ckks_mul_relin_host, the
    headline `e2e`) and limbs packed at their primes' bit widths
    (ckks_mul_relin_host_packed).  The chunk size of each is the fastest of two
    untimed passes at each of 4, 8, 16, 32; the JSON keeps those passes and the
    timed steps one by one."""
    import paper_2506_19693_gb300 as ck
    n = ctx.n
    B = len(A)
    out_level = level - 1
    sa, sb = A[0].scale, Bc[0].scale
    world = 1 if dist is None else dist.get_world_size()
    steps = max(1, min(args.steps, 3))

    def measure(once):
        best, best_t, sel = 16, None, {}
        for chunk in (4, 8, 16, 32):
            once(chunk)  # staging allocated outside the timing
            for _ in range(2):  # the faster of two passes per candidate
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                once(chunk)
                torch.cuda.synchronize()
                t = time.perf_counter() - t0
                sel[chunk] = min(sel.get(chunk, t), t)
                if best_t is None or t < best_t:
                    best, best_t = chunk, t
        torch.cuda.synchronize()
        per_step = []
        for _ in range(steps):  # each call ends synchronised: per-step times cost nothing extra
            t0 = time.perf_counter()
            once(best)
            torch.cuda.synchronize()
            per_step.append(time.perf_counter() - t0)
        total = max_over_ranks([sum(per_step)], dist, "cuda")[0]
        return total, best, {"step_ms": [round(1e3 * t, 3) for t in per_step],
                             "chunk_selection_ms": {c: round(1e3 * t, 3) for c, t in sel.items()}}

    # plain uint64 limbs
    host_a = torch.empty((B, 2, level + 1, n), dtype=torch.int64, pin_memory=True)
    host_b = torch.empty((B, 2, level + 1, n), dtype=torch.int64, pin_memory=True)
    host_out = torch.empty((B, 2, out_level + 1, n), dtype=torch.int64, pin_memory=True)
    for i in range(B):
        host_a[i].copy_(A[i].data[:, : level + 1])
        host_b[i].copy_(Bc[i].data[:, : level + 1])
    dt_raw, chunk_raw, detail_raw = measure(lambda ch: ctx.mul_relin_host(host_a, host_b, sa, sb, level, host_out,
                                                              rescale=ck.RESCALE_MERGED, chunk=ch))
    raw = {"value": world * B * steps / dt_raw, "unit": UNIT, "chunk_pairs": chunk_raw, **detail_raw,
           "h2d_bytes_per_step": 2 * B * 2 * (level + 1) * n * 8,
           "d2h_bytes_per_step": B * 2 * (out_level + 1) * n * 8, "call": "ckks_mul_relin_host"}
    del host_a, host_b, host_out
    # packed limbs (the inputs packed once, untimed, as a user stores them)
    wi, wo = ctx.wire_bytes(level), ctx.wire_bytes(out_level)
    pa = torch.empty(B * wi, dtype=torch.uint8, pin_memory=True)
    pb = torch.empty(B * wi, dtype=torch.uint8, pin_memory=True)
    po = torch.empty(B * wo, dtype=torch.uint8, pin_memory=True)
    for i in range(B):
        ctx.export_packed(A[i], pa[i * wi:(i + 1) * wi])
        ctx.export_packed(Bc[i], pb[i * wi:(i + 1) * wi])
    dt, chunk, detail = measure(lambda ch: ctx.mul_relin_host_packed(pa, pb, sa, sb, level, po,
                                                             rescale=ck.RESCALE_MERGED, chunk=ch))
    packed = {"value": world * B * steps / dt, "unit": UNIT, "chunk_pairs": chunk, **detail,
              "h2d_bytes_per_step": 2 * B * wi,
              "d2h_bytes_per_step": B * wo, "call": "ckks_mul_relin_host_packed (limbs at their primes' bit widths)"}
    # the headline: uint64 limbs.  That pipeline is bound by the host link (both
    # directions at once); the packed one moves 14% fewer bytes but is bound by
    # the products plus its pack/unpack kernels
    return dict(raw, steps=steps, call="ckks_mul_relin_host (page-locked host buffers)",
                clock="host perf_counter around synchronised steps", packed_limbs=packed)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-reboot", action="store_true")
    ap.add_argument("--no-uneven", action="store_true")
    ap.add_argument("--no-iterative", action="store_true")
    ap.add_argument("--no-key-compression", action="store_true")
    ap.add_argument("--no-sparse-boot", action="store_true")
    ap.add_argument("--no-n-scaling", action="store_true")
    ap.add_argument("--no-form-compare", action="store_true")
    ap.add_argument("--no-tc-ntt", action="store_true")
    ap.add_argument("--no-finish-compare", action="store_true")
    ap.add_argument("--form", default="tensor", choices=["uint64", "tensor", "fused"],
                    help="basis conversion on the CUDA cores (uint64), on the tensor cores (tensor), or on the "
                         "CUDA cores fused with the transforms' column passes (fused)")
    ap.add_argument("--small", action="store_true",
                    help="8 pairs and 2 bootstraps: a few GB on the device, for ncu captures")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
