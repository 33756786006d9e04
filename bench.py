"""Throughput of the Schwinger-model HMC hot path on one GB300 (or N, one
process per GPU, chains sharded across ranks: weak scaling).

Workload (the mixed-precision versus FP64 configuration of the 64 x 64
lattice): 64 x 64 sites, beta = 2.0, kappa = 0.26, tau = 1, the adapted
nested force-gradient scheme (outer n = 8, inner m = 2, exact C_FF),
FP32 CG with FP64 reliable updates to a true relative residual of 1e-10;
304 chains per GPU advance one trajectory per step (at least the 200
trajectories per step of the configuration, rounded up to two full waves of
the 152 chains the chain-resident CG holds on the GPU at once; --chains 200
runs exactly 200, a second wave of 48 chains then leaves most SMs idle).
The chains start
from one configuration thermalised by this library's own HMC (untimed);
every step draws fresh momenta and pseudofermion noise (pre-generated on
the device before the timed region).

A "step" is one HMC trajectory of every chain: heatbath, H, the MD
trajectory (all forces, CG solves, force-gradient term, link and momentum
updates), H, Metropolis.  value = trajectories per second over all ranks.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (one chain's trajectory per step).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {
    "workload": "64x64 beta=2.0 kappa=0.26, 304 chains/GPU, adapted nested FG n=8 m=2, "
                "mixed-precision CG tol 1e-10 (1e-12 for the S_F of H)",
    "L": 64, "T": 64, "beta": 2.0, "kappa": 0.26, "chains_per_gpu": 304,
    "scheme": "adapted_nested_fg", "tau": 1.0, "n": 8, "M": 2, "fg": "exact",
    "cg_tol": 1e-10, "cg_tol_action": 1e-12, "cg_delta": 0.0003, "precision": "mixed",
}
# Global-memory bytes per site and CG iteration of a memory-resident CG
# iteration (the grid-wide pair of solver.cu: kernel A reads r, p, U and
# writes p, t; kernel B reads t, U, p, x, r and writes x, r; 16 B each in
# FP32, 32 B in FP64).
CG_BYTES_PER_SITE_ITER = {"mixed": (3 + 2) * 16 + (5 + 2) * 16, "f64": (3 + 2) * 32 + (5 + 2) * 32}
# The fused streaming iteration of large lattices (cg_tiled.cu): F reads r,
# p_old, U and writes p, A p; x += alpha p_old in L2 (read and written back);
# R reads r, A p and writes r.
FUSED_CG_BYTES_PER_SITE_ITER = (3 + 2) * 16 + 2 * 16 + (2 + 1) * 16
# Shared-memory bytes per site and iteration of the chain-resident FP32 CG
# (cg_chain.cu), by kernel variant, in the steady state of a walk (the reads
# that start each thread's strip are left out).  Strided layout (0): p update
# 2 x 16, t = D p reads 5 p + 3 U and writes t (9 x 16), D^dag t reads 5 t +
# 3 U + p (9 x 16).  Column layout (1, 2): the t-neighbour below, its link and
# the site's own value come from registers, the links are split into x and t
# halves and x += alpha p rides on the p update, so D p reads p at x +- 1 and
# t + 1 (3 x 16), U_x, U_t (16) and U_x(n - x) (8) and writes t (16), D^dag t
# the same without the write.  Two-block clusters (3, 4) and the 4-block
# cluster of 128 x 128 chains: the column layout with whole-site links and the
# p read of x += alpha p in the D^dag stage (2 x 6 x 16).  Column pairs (5-7):
# per two sites of a row, D reads 4 spinors (64) and 5 link halves (40) and
# writes 2 (32); D^dag the same without the writes.
SMEM_BYTES_STRIDED = 20 * 16
SMEM_BYTES_COLUMN = 2 * 16 + (4 * 16 + 8 + 16) + (3 * 16 + 8 + 16)
SMEM_BYTES_CLUSTER = 14 * 16
SMEM_BYTES_PAIR = 2 * 16 + (64 + 40 + 32) // 2 + (64 + 40) // 2
SMEM_BYTES_BY_VARIANT = ([SMEM_BYTES_STRIDED] + [SMEM_BYTES_COLUMN] * 2 + [SMEM_BYTES_CLUSTER] * 2
                         + [SMEM_BYTES_PAIR] * 4)
# What actually crosses shared memory per site-iteration where it differs
# from the layout's count: column pairs with x, p and the links in tensor
# memory (8) take the thread's own p in D, its own t in D^dag and its own 4
# link halves from registers and TMEM, so per two sites D reads the two outer
# x-neighbours (32) and one link half (8) and writes 2 (32), D^dag reads 2
# neighbours and one link half, the p update only writes p (16): 72 B.  x,
# p and the links move between TMEM and registers (32 + 32 + 32 B per site
# and iteration, not through shared memory).  The roofline keeps the column
# pairs' 152 B (the operands an iteration consumes from on-chip storage), so
# that the variants compare.
SMEM_TRAFFIC_BY_VARIANT = {8: 16 + (32 + 8 + 32) // 2 + (32 + 8) // 2}
# Shared-memory bandwidth per SM and clock (32 banks x 4 B).
SMEM_BYTES_PER_CLK_PER_SM = 128
NUM_SMS = 152
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# the committed ncu captures, keyed by kernel, with the sources they were
# taken on: a changed source makes the figure stale (reported as null)
NCU_CAPTURES = {
    # the first solve of a step (S_F of H from the cold start, tolerance 1e-12,
    # reliable-update factor 1e-3), one launch of 304 chains
    "k_cg_chain_pair<8,256,64,64,1,true>": {
        "sources": {"paper_1512_03812_gb300/csrc/cg_chain.cu": "8b7d70f02c100029",
                    "paper_1512_03812_gb300/csrc/common.cuh": "e4b4838dd0c85c79"},
        "dram_bytes_per_launch": 250515456 + 265532160},
    "k_cg_chain_pair<8,256,64,64,1>": {
        "sources": {"paper_1512_03812_gb300/csrc/cg_chain.cu": "108bcefb617db4c2",
                    "paper_1512_03812_gb300/csrc/common.cuh": "e4b4838dd0c85c79"},
        "dram_bytes_per_launch": 117513472 + 57990912},
    # back-to-back launches with --cache-control none (the mean of 5 launches):
    # each pays for its predecessor's write-back, as in the bench's timing
    "k_ddagd_stream": {
        "sources": {"paper_1512_03812_gb300/csrc/stream.cuh": "8efeb63c67537b28",
                    "paper_1512_03812_gb300/csrc/ddagd.cu": "53e8616d44d12d34",
                    "paper_1512_03812_gb300/csrc/common.cuh": "e4b4838dd0c85c79"},
        "dram_bytes_per_launch": 134663884 + 68860569},
}


def _sha16(path):
    import hashlib
    with open(os.path.join(ROOT, path), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu capture, or
    None if there is none or its sources have changed."""
    cap = NCU_CAPTURES.get(kernel)
    if cap is None or any(_sha16(p) != h for p, h in cap["sources"].items()):
        return None
    return cap["dram_bytes_per_launch"]


# the chain-resident CG kernels by variant index (sm_set_cg_variant)
CHAIN_KERNELS = ["k_cg_chain_mixed<8,512>", "k_cg_chain_col<8,512>", "k_cg_chain_col<16,256>",
                 "k_cg_chain_cluster<8,256,2>", "k_cg_chain_cluster<4,512,2>",
                 "k_cg_chain_pair<4,512,64,64,1>", "k_cg_chain_pair<8,256,64,64,1>",
                 "k_cg_chain_pair<8,128,64,64,2>", "k_cg_chain_pair<8,256,64,64,1,true>"]


def kappa_to_m0(k):
    return 1.0 / (2.0 * k) - 2.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed
    region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"bench_clocks_{os.getpid()}_{index}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ ranks --------

def shard(world, rank, chains_per_rank):
    """The chains of one rank: an independent batch with its own random
    streams (the path shards as independent chains: weak scaling, no
    data-path collective)."""
    return {"seed": 1234 + 7919 * rank, "chains": chains_per_rank,
            "first_chain": rank * chains_per_rank, "world": world}


def max_over_ranks(x, dist=None, device=None):
    """Max of a per-rank float over all ranks (the only collective)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def aggregate(world, chains_per_rank, steps, ms_max):
    """Whole-job trajectories per second from the slowest rank's time."""
    return world * chains_per_rank * steps / (ms_max / 1e3)


def rank_env():
    """(world size, rank, local rank) of this process (1, 0, 0 when not
    started by torch.distributed.run)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _free_port():
    import socket
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_command(n, argv, port=None):
    """The command that runs this script as n ranks on one node, one process
    per GPU (torch.distributed.run, rendezvous on 127.0.0.1)."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
            f"--nproc-per-node={int(n)}", "--master-addr", "127.0.0.1",
            "--master-port", str(port or _free_port()), os.path.abspath(__file__), *argv]


def launch_ranks(n, argv, capture=False, timeout=None):
    """Starts n ranks of this script with the arguments argv and waits for
    them; returns the completed process (its stdout captured if asked)."""
    return subprocess.run(rank_command(n, argv), capture_output=capture, text=True,
                          timeout=timeout)


def check_world(gpus, world):
    """A run asked for `gpus` ranks must have been started as that many."""
    if world != gpus:
        raise SystemExit(f"bench.py: --gpus {gpus} but WORLD_SIZE is {world}; start it with "
                         f"--gpus {gpus} alone (it launches its ranks) or under "
                         f"torch.distributed.run --nproc-per-node {gpus}")


def check_distinct(dist, key):
    """Every rank reports a different `key` (its device): gathered on all
    ranks, refused if two ranks share one."""
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return [key]
    keys = [None] * dist.get_world_size()
    dist.all_gather_object(keys, key)
    if len(set(keys)) != len(keys):
        raise SystemExit(f"bench.py: ranks share a device: {keys}")
    return keys


def run_rank_selftest(args):
    """The rank logic of a multi-rank run without any GPU work (gloo on the
    CPU): world size against --gpus, distinct local ranks, the shards and
    seeds of the chains, and the max-over-ranks timing and the aggregate."""
    import torch.distributed as dist
    world, rank, local = rank_env()
    check_world(args.gpus, world)
    if world > 1:
        dist.init_process_group("gloo")
    locals_ = check_distinct(dist, local)
    sh = shard(world, rank, args.chains)
    shards = [None] * world
    if world > 1:
        dist.all_gather_object(shards, sh)
    else:
        shards = [sh]
    ms = max_over_ranks(100.0 + 10.0 * rank, dist)
    if rank == 0:
        print(json.dumps({"world": world, "local_ranks": locals_, "shards": shards,
                          "ms_max": ms, "value": aggregate(world, args.chains, 1, ms)}),
              flush=True)
    if world > 1:
        dist.destroy_process_group()


def bench_config(W, chains, world, args):
    """The `config` of the JSON line, the same for both arms."""
    return dict(W, chains_per_gpu=chains, precision=args.prec, parallelism=f"replicas{world}",
                l2="flushed between steps (256 MiB write)", cuda_graph=bool(args.graph))


def thermalise_64(P, dev, W, therm):
    """One 64 x 64 configuration at the workload's couplings, thermalised by
    this library's HMC (untimed): heavy fermions first (kappa 0.10: cheap,
    stable), then the working kappa with small steps, every trajectory
    accepted, then a few with Metropolis."""
    import torch
    L, T = W["L"], W["T"]
    t0 = time.time()
    q1 = torch.zeros((L * T, 2), dtype=torch.float64, device=dev)
    g1 = torch.Generator(device=dev)
    g1.manual_seed(99)
    acc_th = []
    fine = P.CG(1e-8, 20000, "mixed")
    phases = [(0.10, P.MD(scheme="nested_leapfrog", tau=1.0, n=5, M=8, cg=fine), therm, 0.0),
              (W["kappa"], P.MD(scheme="nested_leapfrog", tau=1.0, n=16, M=4, cg=fine),
               therm // 2, 0.0),
              (W["kappa"], P.MD(scheme="nested_leapfrog", tau=1.0, n=16, M=4, cg=fine),
               therm // 4, None)]
    for kap, mdt, ntraj, uforce in phases:
        one = P.Lattice(L, T, W["beta"], kappa_to_m0(kap), device=dev)
        for _ in range(ntraj):
            p = torch.randn((L * T, 2), generator=g1, device=dev, dtype=torch.float64)
            e = torch.view_as_complex(torch.randn((L * T, 2, 2), generator=g1, device=dev,
                                                  dtype=torch.float64) * math.sqrt(0.5))
            u = float(torch.rand(1, generator=g1, device=dev, dtype=torch.float64))
            u = u if uforce is None else uforce
            dH, _, acc = one.hmc_trajectory(q1, p, e.contiguous(), u, mdt, check=False)
            acc_th.append((kap, bool(acc[0]), float(dH[0])))
    log(f"thermalised in {time.time() - t0:.1f}s: " +
        " ".join(f"k{k:.2f}:{'A' if a else 'r'}{d:+.2g}" for k, a, d in acc_th))
    return q1


# ------------------------------------------------------------ our arm ------

def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1512_03812_gb300 as P
    from paper_1512_03812_gb300 import binding

    world, rank, local = rank_env()
    check_world(args.gpus, world)
    if local >= torch.cuda.device_count():
        raise SystemExit(f"bench.py: local rank {local} but {torch.cuda.device_count()} GPUs")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    props = torch.cuda.get_device_properties(dev)
    check_distinct(dist, str(getattr(props, "uuid", local)))
    P.build()

    W = WORKLOAD
    B, L, T = args.chains, W["L"], W["T"]
    m0 = kappa_to_m0(W["kappa"])
    lat = P.Lattice([L] * B, [T] * B, W["beta"], m0, device=dev)
    N = lat.N
    W = dict(W, n=args.n, M=args.M, cg_delta=args.delta)
    if args.sf_start != "solve":
        W["sf_start"] = args.sf_start
    cgp = P.CG(tol=W["cg_tol"], maxit=20000, prec=args.prec, delta=args.delta, algo=args.algo)
    md = P.MD(scheme=W["scheme"], tau=W["tau"], n=W["n"], M=W["M"], fg=W["fg"], cg=cgp,
              tol_action=W["cg_tol_action"], sf_start=args.sf_start)
    gen = torch.Generator(device=dev)
    gen.manual_seed(shard(world, rank, B)["seed"])

    def draws(k):
        p = torch.randn((k, N, 2), generator=gen, device=dev, dtype=torch.float64)
        e = torch.randn((k, N, 2, 2), generator=gen, device=dev, dtype=torch.float64)
        e = torch.view_as_complex(e * math.sqrt(0.5)).contiguous()
        u = torch.rand((k, B), generator=gen, device=dev, dtype=torch.float64).cpu().numpy()
        return p, e, u

    q1 = thermalise_64(P, dev, W, args.therm)
    q_start = q1.repeat(B, 1).contiguous()

    flush = torch.empty(int(256 * 2 ** 20), dtype=torch.uint8, device=dev)

    # pick the chain-resident CG kernel for this batch (untimed): time every
    # applicable variant on one representative solve at the start links
    tune = None
    if args.cg_variant >= 0:
        lat.set_cg_variant(args.cg_variant)
        tune = {"variant": args.cg_variant, "pinned": True}
    elif args.prec == "mixed" and args.algo != "grid":
        U64s, U32s = lat.links(q_start)
        b_t = torch.view_as_complex(torch.randn((N, 2, 2), generator=gen, device=dev,
                                                dtype=torch.float64)).contiguous()
        v, vms = lat.autotune_cg(U64s, U32s, b_t, cgp)
        tune = {"variant": v, "ms_per_variant": [round(t, 3) for t in vms],
                "variants": ["strided 512x8", "column 512x8", "column 256x16",
                             "column 2-block cluster 256x8", "column 2-block cluster 512x4",
                             "column pairs 512x2x4", "column pairs 256x2x8",
                             "column pairs 2-block cluster 128x2x8",
                             "column pairs 256x2x8, x in TMEM"]}
        log(f"autotuned chain CG: variant {v}, ms {vms}")
        del U64s, U32s, b_t

    # (the graph keeps the kernel variants chosen when it is captured)
    graph = None
    if args.graph:
        # one captured trajectory bound to fixed buffers; a step refills them
        p_buf = torch.empty((N, 2), dtype=torch.float64, device=dev)
        e_buf = torch.empty((N, 2), dtype=torch.complex128, device=dev)
        q_buf = q_start.clone()
        graph = lat.hmc_graph(q_buf, p_buf, e_buf, md)

    def step(q, p, e, u):
        flush.fill_(1)  # evict the previous step's working set from L2
        if graph is None:
            return lat.hmc_trajectory(q, p, e, u, md, check=False)
        q_buf.copy_(q)
        p_buf.copy_(p)
        e_buf.copy_(e)
        r = graph.run(u)
        q.copy_(q_buf)
        return r

    q = q_start.clone()
    pw, ew, uw = draws(args.warmup)
    for i in range(args.warmup):
        step(q, pw[i], ew[i], uw[i])
    torch.cuda.synchronize()
    del pw, ew
    K = args.steps
    pk, ek, uk = draws(K)
    dHs, accs = [], []
    binding.profile_enable(True)
    binding.profile_read(reset=True)
    n0 = binding.launch_count()
    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    for i in range(K):
        torch.cuda.nvtx.range_push("timed_step")  # lets ncu select the timed steps
        dH, _, acc = step(q, pk[i], ek[i], uk[i])
        torch.cuda.nvtx.range_pop()
        dHs.append(dH)
        accs.append(acc)
    st = lat.stats.as_dict()
    ev1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    launches = binding.launch_count() - n0
    prof = binding.profile_read(reset=True)
    log(f"timed {K} steps: {ms / K:.1f} ms/step, last-step stats {st}, "
        f"dH[:8] {np.round(dHs[-1][:8], 4)}")
    binding.profile_enable(False)
    ms_max = max_over_ranks(ms, dist, dev)
    traj_per_s = aggregate(world, B, K, ms_max)
    acc_rate = float(np.mean(np.concatenate(accs)))

    # end to end through the public API with host buffers: per step the
    # momenta and noise go host -> device, Delta H and the decisions come back.
    # The copies of step i + 1's inputs run on a copy stream into the other
    # of two device buffers while step i computes (that buffer's last reader,
    # step i - 1, has returned its results to the host); every step's copy
    # lies inside the timed region.
    ph = pk[:K].cpu().pin_memory()
    eh = ek[:K].cpu().pin_memory()
    pd = [torch.empty_like(pk[0]) for _ in range(2)]
    ed = [torch.empty_like(ek[0]) for _ in range(2)]
    ready = [torch.cuda.Event() for _ in range(2)]
    cur = torch.cuda.current_stream(dev)
    cs = torch.cuda.Stream(device=dev)

    def h2d_copy(i):
        with torch.cuda.stream(cs):
            pd[i % 2].copy_(ph[i], non_blocking=True)
            ed[i % 2].copy_(eh[i], non_blocking=True)
            ready[i % 2].record(cs)

    q = q_start.clone()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    cs.wait_stream(cur)
    h2d_copy(0)
    for i in range(K):
        cur.wait_event(ready[i % 2])
        if i + 1 < K:
            h2d_copy(i + 1)
        step(q, pd[i % 2], ed[i % 2], uk[i])
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    h2d = int(pd[0].numel() * 8 + ed[0].numel() * 16 + B * 8)
    d2h = int(B * (8 + 8 + 4))

    # FP64 path on the same inputs: Delta H deviation and throughput
    def md_with(prec, tol, algo=None, variant=None):
        return P.MD(scheme=W["scheme"], tau=W["tau"], n=W["n"], M=W["M"], fg=W["fg"],
                    cg=P.CG(tol=tol, maxit=50000, prec=prec, algo=algo or args.algo,
                            delta=args.delta),
                    tol_action=min(tol, W["cg_tol_action"]), sf_start=args.sf_start)

    def compare(md_a, md_b, steps, time_a=True, time_b=True, lat_b=None):
        """Both arms from q_start on the same momenta, noise and uniforms,
        `steps` trajectories each (the chains of arm b are reset to arm a's
        after every trajectory, so both take the same path); per arm the
        event-timed trajectories/s (flushed L2, as in the timed steps)."""
        lb = lat_b or lat
        qa, qb = q_start.clone(), q_start.clone()
        dev_max, same, ta, tb, acc_a, acc_b = 0.0, [], 0.0, 0.0, [], []
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        for i in range(steps):
            flush.fill_(1)
            f0.record()
            da, _, aa = lat.hmc_trajectory(qa, pk[i], ek[i], uk[i], md_a, check=False)
            f1.record()
            torch.cuda.synchronize()
            ta += f0.elapsed_time(f1)
            flush.fill_(1)
            f0.record()
            db, _, ab = lb.hmc_trajectory(qb, pk[i], ek[i], uk[i], md_b, check=False)
            f1.record()
            torch.cuda.synchronize()
            tb += f0.elapsed_time(f1)
            ok = np.isfinite(da) & np.isfinite(db)
            if ok.any():
                dev_max = max(dev_max, float(np.abs(da[ok] - db[ok]).max()))
            same.append(aa == ab)
            acc_a.append(aa)
            acc_b.append(ab)
            qb.copy_(qa)
        n = world * B * steps
        return {"traj_per_s_a": n / (ta / 1e3) if time_a else None,
                "traj_per_s_b": n / (tb / 1e3) if time_b else None,
                "max_abs_dH_diff": dev_max,
                "same_decisions": float(np.mean(np.concatenate(same))),
                "acc_a": float(np.mean(np.concatenate(acc_a))),
                "acc_b": float(np.mean(np.concatenate(acc_b))), "steps": steps,
                "trajectories_per_arm": n}

    fp64 = None
    if args.fp64_steps > 0:
        # at the workload's tolerance: FP64 (a) against mixed (b)
        r = compare(md_with("f64", W["cg_tol"]), md, args.fp64_steps)
        fp64 = {"traj_per_s": r["traj_per_s_a"], "traj_per_s_mixed_same_inputs": r["traj_per_s_b"],
                "acc": r["acc_a"], "acc_mixed_same_inputs": r["acc_b"],
                "same_decisions": r["same_decisions"],
                "max_abs_dH_mixed_minus_fp64": r["max_abs_dH_diff"], "steps": args.fp64_steps,
                "cg_tol": W["cg_tol"]}
        log(f"fp64 at {W['cg_tol']}: {r}")
        # the deviation any two correct solvers show at this tolerance: FP64
        # chain-resident against FP64 grid-wide (other reduction order, other
        # iterates), and two kernel variants of the mixed solver
        r = compare(md_with("f64", W["cg_tol"], algo="chain"), md_with("f64", W["cg_tol"], algo="grid"),
                    1, time_a=False, time_b=False)
        fp64["floor_f64_chain_vs_f64_grid"] = {"cg_tol": W["cg_tol"],
                                               "max_abs_dH_diff": r["max_abs_dH_diff"],
                                               "same_decisions": r["same_decisions"],
                                               "trajectories": r["trajectories_per_arm"]}
        log(f"floor f64 chain vs grid: {r}")
        if tune and not tune.get("pinned"):
            alt = 2 if tune["variant"] != 2 else 1
            lat2 = P.Lattice([L] * B, [T] * B, W["beta"], m0, device=dev)
            lat2.set_cg_variant(alt)
            r = compare(md, md, 1, time_a=False, time_b=False, lat_b=lat2)
            fp64["floor_mixed_variant_%d_vs_%d" % (tune["variant"], alt)] = {
                "cg_tol": W["cg_tol"], "max_abs_dH_diff": r["max_abs_dH_diff"],
                "same_decisions": r["same_decisions"], "trajectories": r["trajectories_per_arm"]}
            log(f"floor mixed variants: {r}")
            del lat2
    if args.tight_tol > 0 and args.tight_steps > 0:
        # both paths timed at the tolerance at which their Delta H agree
        # within 1e-8: FP64 (a) against mixed (b), MD and action solves at
        # tight_tol
        r = compare(md_with("f64", args.tight_tol), md_with("mixed", args.tight_tol),
                    args.tight_steps)
        tight = {"cg_tol": args.tight_tol, "cg_tol_action": min(args.tight_tol, W["cg_tol_action"]),
                 "traj_per_s_fp64": r["traj_per_s_a"], "traj_per_s_mixed": r["traj_per_s_b"],
                 "mixed_over_fp64": r["traj_per_s_b"] / r["traj_per_s_a"],
                 "max_abs_dH_mixed_minus_fp64": r["max_abs_dH_diff"],
                 "same_decisions": r["same_decisions"], "acc_fp64": r["acc_a"],
                 "acc_mixed": r["acc_b"], "steps": r["steps"],
                 "trajectories_per_arm": r["trajectories_per_arm"],
                 "target_dH_within": 1e-8,
                 "meets_target": bool(r["max_abs_dH_diff"] <= 1e-8 and r["same_decisions"] == 1.0)}
        log(f"tight tol {args.tight_tol}: {tight}")
        fp64 = dict(fp64 or {}, tight_tol=tight)

    # roofline of the dominant kernel: the CG solve.  The chain-resident form
    # (every chain of this workload fits) keeps U, p, t in shared memory and
    # x, r in registers, so its bound is shared-memory bandwidth, not HBM.
    peaks, src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    bps = CG_BYTES_PER_SITE_ITER[args.prec]
    ksec = prof["iter_ms"] / 1e3
    hbm_eq = bps * prof["site_iters"] / ksec / 1e9 if ksec else 0.0
    chain = args.algo == "chain" or (args.algo == "auto" and args.prec == "mixed")
    rates = binding.measure_peaks()
    if chain and args.prec == "mixed":
        f_mhz = (clk or {}).get("sm_mhz") or 2070.0
        nominal = NUM_SMS * SMEM_BYTES_PER_CLK_PER_SM * f_mhz * 1e6 / 1e9
        peak = rates["smem_read_gbs"]
        var = tune["variant"] if tune else 0
        sbytes = SMEM_BYTES_BY_VARIANT[var]
        ach = sbytes * prof["site_iters"] / ksec / 1e9 if ksec else 0.0
        kname = CHAIN_KERNELS[var]
        roofline = {"bound": "smem", "kernel": kname + " (chain-resident CG)",
                    "achieved": round(ach, 1), "peak": round(peak, 1), "unit": "GB/s",
                    "frac": round(ach / peak, 4),
                    "peak_source": "measured in this run (sm_peak_smem_read: 16-byte shared "
                                   "loads on every SM)",
                    "peak_nominal": round(nominal, 1),
                    "peak_nominal_source": f"{NUM_SMS} SMs x {SMEM_BYTES_PER_CLK_PER_SM} B/clk x "
                                           f"{f_mhz:.0f} MHz (median SM clock under load)",
                    "bytes_per_site_iter": sbytes,
                    "smem_bytes_per_site_iter": SMEM_TRAFFIC_BY_VARIANT.get(var, sbytes),
                    "traffic": ncu_traffic(kname), "traffic_unit": "DRAM bytes per launch (ncu)",
                    "hbm_equivalent": {"achieved": round(hbm_eq, 1), "peak": hbm,
                                       "unit": "GB/s", "frac": round(hbm_eq / hbm, 4),
                                       "bytes_per_site_iter": bps, "peak_source": src}}
    else:
        roofline = {"bound": "hbm", "kernel": "cg iteration (k_cg_a + k_cg_b)",
                    "achieved": round(hbm_eq, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(hbm_eq / hbm, 4), "peak_source": src, "traffic": None,
                    "bytes_per_site_iter": bps}
    roofline.update({"site_iters": prof["site_iters"], "kernel_ms": round(prof["iter_ms"], 3),
                     "kernel_share_of_step": round(prof["iter_ms"] / ms, 4)})

    ddagd = None
    if not args.no_ddagd:
        ddagd = {"f32": measure_ddagd(torch, P, dev, prec="f32"),
                 "f64": measure_ddagd(torch, P, dev, prec="f64", rates=rates)}
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu:
        # the oracle on the host cores, from the same thermalised start with
        # the first timed step's momenta, noise and uniforms
        qh = q_start[:L * T].cpu().numpy()
        ph, eh = pk[0].cpu().numpy(), ek[0].cpu().numpy()
        jobs = [(qh, ph[c * L * T:(c + 1) * L * T], eh[c * L * T:(c + 1) * L * T], float(uk[0][c]))
                for c in range(B)]
        cpu = cpu_baseline(jobs)
    out = {
        "metric": "HMC trajectories/s", "value": round(traj_per_s, 3),
        "unit": "trajectories/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": round(ms_max / K, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.prec == "mixed" else "f64",
        "data": "synthetic (own thermalised start, seeded momenta/noise)",
        "config": bench_config(W, B, world, args),
        "cg_autotune": tune,
        "acceptance": round(acc_rate, 4),
        "e2e": {"value": round(aggregate(world, B, K, e2e_ms), 3), "unit": "trajectories/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "fp64": fp64,
        "ddagd_2048": ddagd,
        "measured_rates": rates,
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    print(json.dumps(out), flush=True)


# ------------------------------------------- the other two configurations --

OTHER_WORKLOADS = {
    "batched": {
        "workload": "256 chains, sides from {16,32,48,64,128}, beta in {1,2,4}, kappa in "
                    "[0.20,0.26], adapted nested FG n=6 m=2, mixed CG tol 1e-10",
        "chains": 256, "scheme": "adapted_nested_fg", "tau": 1.0, "n": 6, "M": 2,
        "cg_tol": 1e-10, "cg_tol_action": 1e-12, "cg_delta": 0.001, "therm": (6, 4)},
    "large": {
        "workload": "2048x2048 beta=8.0 kappa=0.255, adapted nested FG n=8 m=3, mixed CG tol 1e-10",
        "L": 2048, "beta": 8.0, "kappa": 0.255, "scheme": "adapted_nested_fg", "tau": 1.0,
        "n": 8, "M": 3, "cg_tol": 1e-10, "cg_tol_action": 1e-12, "cg_delta": 0.001,
        "therm": (3, 2)},
}


BATCHED_KERNELS = {16: "k_cg_chain_pair<2,64,16,16,1>", 32: "k_cg_chain_pair<4,128,32,32,1>",
                   48: "k_cg_chain_pair<4,288,48,48,1>", 64: "k_cg_chain_pair<8,256,64,64,1,true>",
                   128: "k_cg_chain_pair<4,256,128,128,8,true> (8-block clusters)"}


def batched_kernels(torch, P, lat, q, Ls, betas, m0, cgp, smem_peak):
    """The shape groups' kernels one at a time: each group's chains as a
    lattice of their own with the batch's current links, one solve of a
    seeded right-hand side timed with CUDA events after a warm-up solve, and
    the group's shared-memory bytes (152 per site-iteration) over that time.
    The longest chain of a group sets its launch's duration, so the mean and
    largest iteration counts are given beside it."""
    g = torch.Generator(device=lat.device)
    g.manual_seed(77)
    out = []
    off = lat.offsets
    U64, U32 = lat.links(q)
    b = torch.view_as_complex(torch.randn((lat.N, 2, 2), generator=g, device=lat.device,
                                          dtype=torch.float64)).contiguous()
    for side in sorted(set(Ls)):
        idx = [c for c in range(len(Ls)) if Ls[c] == side]
        rows = torch.tensor(np.concatenate([np.arange(off[c], off[c + 1]) for c in idx]),
                            device=lat.device)
        sub = P.Lattice([side] * len(idx), [side] * len(idx), np.asarray(betas)[idx],
                        np.asarray(m0)[idx], device=lat.device)
        u64, u32, bs = U64[rows].contiguous(), U32[rows].contiguous(), b[rows].contiguous()
        sub.cg_solve(u64, u32, bs, cgp)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        _, its, _ = sub.cg_solve(u64, u32, bs, cgp)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        si = int(np.sum(its)) * side * side
        gbs = SMEM_BYTES_PAIR * si / (ms / 1e3) / 1e9
        out.append({"side": side, "kernel": BATCHED_KERNELS.get(side, "k_cg_chain_mixed"),
                    "chains": len(idx), "ms_per_solve": round(ms, 3), "site_iters": si,
                    "iters_mean": round(float(np.mean(its)), 1), "iters_max": int(np.max(its)),
                    "bytes_per_site_iter": SMEM_BYTES_PAIR, "achieved": round(gbs, 1),
                    "frac": round(gbs / smem_peak, 4)})
        del sub
    return out


def run_other(args):
    """Trajectory throughput of the batched-chain or the large-lattice
    configuration (one JSON line; thermalisation untimed, as for the
    default workload)."""
    import torch

    import paper_1512_03812_gb300 as P
    from paper_1512_03812_gb300 import binding
    from paper_1512_03812_gb300 import inputs as I
    spec = OTHER_WORKLOADS[args.workload]
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    P.build()
    if args.workload == "batched":
        n = spec["chains"]
        sides = I.chain_sides(n, 81)
        betas, kappas = I.chain_couplings(n, 82)
        Ls = Ts = [int(s) for s in sides]
    else:
        Ls = Ts = [spec["L"]]
        betas, kappas = np.array([spec["beta"]]), np.array([spec["kappa"]])
    m0 = np.array([kappa_to_m0(k) for k in kappas])
    lat = P.Lattice(Ls, Ts, betas, m0, device=dev)
    N, B = lat.N, lat.nchains
    g = torch.Generator(device=dev)
    g.manual_seed(4321)

    def draw():
        p = torch.randn((N, 2), generator=g, device=dev, dtype=torch.float64)
        e = torch.view_as_complex(torch.randn((N, 2, 2), generator=g, device=dev,
                                              dtype=torch.float64) * math.sqrt(0.5)).contiguous()
        u = torch.rand(B, generator=g, device=dev, dtype=torch.float64).cpu().numpy()
        return p, e, u

    fine = P.CG(1e-8, 50000, "mixed", delta=args.delta)
    q = torch.zeros((N, 2), dtype=torch.float64, device=dev)
    heavy = P.Lattice(Ls, Ts, betas, np.full(B, kappa_to_m0(0.10)), device=dev)
    t0 = time.time()
    for _ in range(spec["therm"][0]):
        p, e, _ = draw()
        heavy.hmc_trajectory(q, p, e, np.zeros(B),
                             P.MD(scheme="nested_leapfrog", tau=1.0, n=5, M=8, cg=fine), check=False)
    for _ in range(spec["therm"][1]):
        p, e, _ = draw()
        lat.hmc_trajectory(q, p, e, np.zeros(B),
                           P.MD(scheme="nested_leapfrog", tau=1.0, n=16, M=4, cg=fine), check=False)
    del heavy
    log(f"{args.workload}: thermalised in {time.time() - t0:.1f}s")
    cgp = P.CG(tol=spec["cg_tol"], maxit=50000, prec="mixed", delta=args.delta, algo=args.algo)
    md = P.MD(scheme=spec["scheme"], tau=spec["tau"], n=spec["n"], M=spec["M"], cg=cgp,
              tol_action=spec["cg_tol_action"])
    flush = torch.empty(int(256 * 2 ** 20), dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        p, e, u = draw()
        flush.fill_(1)
        lat.hmc_trajectory(q, p, e, u, md, check=False)
    draws = [draw() for _ in range(args.steps)]
    # the batched configuration replays its trajectory as a CUDA graph (every
    # solve is chain-resident); the eager steps after it give the CG kernel
    # times (solves inside a graph are not timed) and the eager throughput
    use_graph = args.workload == "batched"
    graph = None
    if use_graph:
        p_buf = torch.empty((N, 2), dtype=torch.float64, device=dev)
        e_buf = torch.empty((N, 2), dtype=torch.complex128, device=dev)
        q_buf = q.clone()
        graph = lat.hmc_graph(q_buf, p_buf, e_buf, md)
        for _ in range(args.warmup):
            p, e, u = draw()
            p_buf.copy_(p)
            e_buf.copy_(e)
            graph.run(u)

    def timed(eager):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        accs = []
        for p, e, u in draws:
            flush.fill_(1)
            torch.cuda.nvtx.range_push("timed_step")  # lets ncu select the timed steps
            if eager:
                _, _, acc = lat.hmc_trajectory(q, p, e, u, md, check=False)
            else:
                p_buf.copy_(p)
                e_buf.copy_(e)
                _, _, acc = graph.run(u)
            torch.cuda.nvtx.range_pop()
            accs.append(acc)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), accs

    n0 = binding.launch_count()
    clocks = Clocks(0)
    clocks.start()
    if use_graph:
        ms, accs = timed(False)
        graph_launches = int(binding.launch_count() - n0)
    binding.profile_enable(True)
    binding.profile_read(reset=True)
    ms_eager, accs_eager = timed(True)
    clk = clocks.stop()
    if not use_graph:
        ms, accs = ms_eager, accs_eager
        graph_launches = int(binding.launch_count() - n0)
    prof = binding.profile_read(reset=True)
    binding.profile_enable(False)
    # the roofline's share is that of the eager steps, whose kernels it timed
    ms_share = ms_eager
    st = lat.stats.as_dict()
    peaks, src = measured_peaks()
    rates = binding.measure_peaks()
    ksec = prof["iter_ms"] / 1e3
    bps = CG_BYTES_PER_SITE_ITER["mixed"]
    hbm = float(peaks["hbm_gbs"])
    ach = bps * prof["site_iters"] / ksec / 1e9 if ksec else 0.0
    common = {"site_iters": prof["site_iters"], "kernel_ms": round(prof["iter_ms"], 2),
              "res_ms": round(prof["res_ms"], 2),
              "kernel_share_of_step": round(prof["iter_ms"] / ms_share, 4), "traffic": None,
              "timed_on": "eager steps" if use_graph else "the timed steps"}
    if args.workload == "batched":
        # every chain is chain-resident: the iteration data stays in shared
        # memory, so the bound is shared-memory bandwidth (HBM-equivalent
        # bytes beside it for context).  Every shape of this batch has a
        # column-pair kernel (152 B per site-iteration): 16, 32, 48 and 64
        # one block per chain, 128 x 128 8-block clusters
        sach = SMEM_BYTES_PAIR * prof["site_iters"] / ksec / 1e9 if ksec else 0.0
        roofline = dict({"bound": "smem",
                         "kernel": "chain-resident CG (one launch per shape group: column pairs "
                                   "16x16, 32x32, 48x48, 64x64 one block per chain; 128x128 "
                                   "8-block clusters)",
                         "achieved": round(sach, 1), "peak": round(rates["smem_read_gbs"], 1),
                         "unit": "GB/s", "frac": round(sach / rates["smem_read_gbs"], 4),
                         "peak_source": "measured in this run (sm_peak_smem_read)",
                         "bytes_per_site_iter": SMEM_BYTES_PAIR,
                         "hbm_equivalent": {"achieved": round(ach, 1), "peak": hbm,
                                            "frac": round(ach / hbm, 4),
                                            "bytes_per_site_iter": bps, "peak_source": src},
                         "per_kernel": batched_kernels(torch, P, lat, q, Ls, betas, m0, cgp,
                                                       rates["smem_read_gbs"])},
                        **common)
    else:
        # the 2048^2 lattice takes the fused streaming iteration: F reads r,
        # p_old, U and writes p, A p (80 B), advances x in L2 (32 B of DRAM
        # traffic), R reads r, A p and writes r (48 B)
        fbps = FUSED_CG_BYTES_PER_SITE_ITER
        fach = fbps * prof["site_iters"] / ksec / 1e9 if ksec else 0.0
        roofline = dict({"bound": "hbm",
                         "kernel": "fused streaming CG iteration (k_cgt_f + k_cgt_r)",
                         "achieved": round(fach, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(fach / hbm, 4), "peak_source": src,
                         "bytes_per_site_iter": fbps}, **common)
    print(json.dumps({
        "metric": "HMC trajectories/s", "value": round(B * args.steps / (ms / 1e3), 4),
        "unit": "trajectories/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (own thermalised start)",
        "config": dict({k: v for k, v in spec.items() if k != "therm"}, sites=N, chains=B,
                       cg_delta=args.delta, l2="flushed between steps (256 MiB write)"),
        "acceptance": round(float(np.mean(np.concatenate(accs))), 4),
        "cuda_graph": use_graph,
        "eager_value": round(B * args.steps / (ms_eager / 1e3), 4) if use_graph else None,
        "last_step_stats": st, "gpu_launches": graph_launches,
        "roofline": roofline, "measured_rates": rates,
        "clocks": clk}), flush=True)


# ------------------------- mixed against FP64 over step sizes (64 x 64) ------

SWEEP = {
    "workload": "64x64 beta=2.0 kappa=0.26, 200 momentum sets from one thermalised "
                "configuration per point, tau=1, outer n in {4,6,8,10}, inner m in {1,2,4} "
                "(nested schemes), plus n in {16,24} for the order in h, mixed CG (FP32 + FP64 "
                "reliable updates) against FP64 CG, "
                "tol 1e-10 (1e-12 for the S_F of H)",
    "chains": 200, "n": (4, 6, 8, 10), "M": (1, 2, 4),
    # larger n for the order of Delta H in h (at n <= 10 most schemes are at or
    # beyond their stability limit on this configuration)
    "n_order": (16, 24),
    "schemes": [("leapfrog", None), ("five_stage", "2mn"), ("five_stage_fg", None),
                ("nested_leapfrog", None), ("nested_fg", None), ("adapted_nested_fg", None)],
}


def _slope(hs, ys):
    """Least-squares slope of log y against log h (the order of Delta H in h)."""
    ok = [(h, y) for h, y in zip(hs, ys) if y and y > 0 and math.isfinite(y)]
    if len(ok) < 2:
        return None
    x = np.log([h for h, _ in ok])
    y = np.log([v for _, v in ok])
    return float(np.polyfit(x, y, 1)[0])


def run_sweep(args):
    """The mixed-precision against FP64 configuration over step sizes: for
    every scheme, outer n and (nested schemes) inner m, one batch of 200
    chains from the same thermalised configuration with fresh momenta and
    noise, once with the mixed CG and once with the FP64 CG on the same
    inputs: acceptance, <|Delta H|>, max |Delta H_mixed - Delta H_FP64| and
    the decisions; then the slope of <|Delta H|> against h per scheme and m
    for both paths.  Writes the JSON to --out as well as to stdout."""
    import torch

    import paper_1512_03812_gb300 as P
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    P.build()
    W = dict(WORKLOAD)
    L, T, B = W["L"], W["T"], SWEEP["chains"]
    q1 = thermalise_64(P, dev, W, args.therm)
    lat = P.Lattice([L] * B, [T] * B, W["beta"], kappa_to_m0(W["kappa"]), device=dev)
    N = lat.N
    qb = q1.repeat(B, 1).contiguous()
    g = torch.Generator(device=dev)
    g.manual_seed(2604)
    cg_m = P.CG(tol=W["cg_tol"], maxit=50000, prec="mixed", delta=args.delta)
    cg_d = P.CG(tol=W["cg_tol"], maxit=50000, prec="f64")
    rows = []
    t_m = t_d = 0.0
    t0 = time.time()
    for scheme, variant in SWEEP["schemes"]:
        Ms = SWEEP["M"] if "nested" in scheme else (1,)
        lam = P.LAMBDA_2MN if variant == "2mn" else 1.0 / 6.0
        for M in Ms:
            for n in SWEEP["n"] + SWEEP["n_order"]:
                p = torch.randn((N, 2), generator=g, device=dev, dtype=torch.float64)
                e = torch.view_as_complex(torch.randn((N, 2, 2), generator=g, device=dev,
                                                      dtype=torch.float64) * math.sqrt(0.5))
                e = e.contiguous()
                u = torch.rand(B, generator=g, device=dev, dtype=torch.float64).cpu().numpy()
                out = {}
                for name, cg in (("mixed", cg_m), ("fp64", cg_d)):
                    md = P.MD(scheme=scheme, tau=W["tau"], n=n, M=M, lam=lam, fg=W["fg"], cg=cg,
                              tol_action=W["cg_tol_action"])
                    q = qb.clone()
                    torch.cuda.synchronize()
                    ta = time.time()
                    dH, _, acc = lat.hmc_trajectory(q, p, e, u, md, check=False)
                    dt = time.time() - ta
                    if name == "mixed":
                        t_m += dt
                    else:
                        t_d += dt
                    out[name] = (dH, acc, dt)
                dm, am, _ = out["mixed"]
                dd, ad, _ = out["fp64"]
                ok = np.isfinite(dm) & np.isfinite(dd)
                row = {"scheme": scheme + ("_2mn" if variant == "2mn" else ""), "n": n,
                       "h": W["tau"] / n, "M": M if "nested" in scheme else None}
                for name, (dH, acc, dt) in out.items():
                    f = np.isfinite(dH)
                    row[name] = {"acceptance": float(np.mean(acc)),
                                 "mean_abs_dH": float(np.abs(dH[f]).mean()) if f.any() else None,
                                 "median_abs_dH": float(np.median(np.abs(dH[f]))) if f.any() else None,
                                 "nonfinite": int((~f).sum()), "seconds": round(dt, 3)}
                row["max_abs_dH_mixed_minus_fp64"] = (float(np.abs(dm[ok] - dd[ok]).max())
                                                      if ok.any() else None)
                row["same_decisions"] = float(np.mean(am == ad))
                rows.append(row)
                log(f"sweep {row['scheme']} n={n} M={M}: acc {row['mixed']['acceptance']:.3f}/"
                    f"{row['fp64']['acceptance']:.3f} dev {row['max_abs_dH_mixed_minus_fp64']:.2e}")
    # the order of Delta H in h from the points inside the stability region
    # (median |Delta H| below 1: beyond it |Delta H| grows exponentially
    # and no power law holds)
    slopes = []
    keys = sorted({(r["scheme"], r["M"]) for r in rows}, key=str)
    for sch, M in keys:
        rs = [r for r in rows if r["scheme"] == sch and r["M"] == M]
        st = {}
        for name in ("mixed", "fp64"):
            ok = [r for r in rs if r[name]["median_abs_dH"] is not None
                  and r[name]["median_abs_dH"] < 1.0]
            st[name] = (_slope([r["h"] for r in ok], [r[name]["median_abs_dH"] for r in ok]),
                        [r["n"] for r in ok])
        slopes.append({"scheme": sch, "M": M, "slope_mixed": st["mixed"][0],
                       "slope_fp64": st["fp64"][0], "fitted_n": st["fp64"][1]})
    devs = [r["max_abs_dH_mixed_minus_fp64"] for r in rows
            if r["max_abs_dH_mixed_minus_fp64"] is not None]
    devs_stable = [r["max_abs_dH_mixed_minus_fp64"] for r in rows
                   if r["max_abs_dH_mixed_minus_fp64"] is not None
                   and (r["fp64"]["median_abs_dH"] or 1e9) < 1.0]
    res = {"metric": "mixed against FP64 over step sizes", "workload": SWEEP["workload"],
           "data": "synthetic (own thermalised start, seeded momenta/noise)",
           "chains": B, "cg_tol": W["cg_tol"], "cg_tol_action": W["cg_tol_action"],
           "cg_delta": args.delta,
           "trajectories_per_path": B * len(rows),
           "wall_s": {"mixed": round(t_m, 2), "fp64": round(t_d, 2),
                      "fp64_over_mixed": round(t_d / t_m, 2) if t_m else None,
                      "total": round(time.time() - t0, 1)},
           "max_abs_dH_mixed_minus_fp64_overall": max(devs) if devs else None,
           "max_abs_dH_mixed_minus_fp64_stable_points": max(devs_stable) if devs_stable else None,
           "same_decisions_overall": float(np.mean([r["same_decisions"] for r in rows])),
           "slope_of_median_abs_dH_in_h": slopes, "points": rows}
    line = json.dumps(res)
    if args.out:
        with open(args.out, "w") as f:
            f.write(json.dumps(res, indent=1) + "\n")
    print(line, flush=True)


# ------------------------------------- the paper's own numerical experiment --

# Sec. 5 of the paper: a 32 x 32 lattice, beta = 1.0, m0 = -0.231367, one
# thermalised configuration, 200 sets of momenta per integrator and step
# size, trajectories of length tau = 2, micro step h / 10 for the nested
# schemes (M = 5 inner leapfrog steps per half macro step).  Table 1 lists the
# step size of each integrator at 90 % acceptance and its inversions of D.
PAPER = {
    "L": 32, "T": 32, "beta": 1.0, "m0": -0.231367, "tau": 2.0, "sets": 200, "M": 5,
    "cg_delta": 0.001,
    # integrator, force-gradient form, Table 1 step size, its D^-1 per step
    # and per trajectory as printed
    "table1": [("five_stage", "exact", 0.0294, 6, 420),
               ("nested_five_stage", "exact", 0.0286, 6, 408),
               ("five_stage_fg", "exact", 0.0550, 10, 370),
               ("five_stage_fg", "shifted", 0.0540, 8, 290),
               ("nested_fg", "exact", 0.0560, 8, 285),
               ("adapted_nested_fg", "exact", 0.0560, 8, 285),
               ("eleven_stage", "exact", 0.0625, 12, 384)],
    # |Delta H| against h (Fig. 1) for every integrator
    "scan_h": (0.0125, 0.025, 0.05, 0.1),
    # the three-level adapted scheme: heavy mass shifts and heavy steps per
    # middle block tried
    "heavy_dm": (0.2, 0.5, 1.0), "M2": (1, 2),
    "scan": [("leapfrog", "exact"), ("nested_leapfrog", "exact"), ("five_stage", "exact"),
             ("nested_five_stage", "exact"), ("five_stage_fg", "exact"),
             ("five_stage_fg", "shifted"), ("nested_fg", "exact"), ("adapted_nested_fg", "exact"),
             ("eleven_stage", "exact")],
}


def run_paper(args):
    """The paper's experiment on this library: Table 1 (acceptance, |Delta H|
    and inversions of D per trajectory at the printed step sizes) and the
    |Delta H| against h scan of Fig. 1, 200 momentum sets each, as one batch
    of 200 chains started from the same thermalised configuration."""
    import torch

    import paper_1512_03812_gb300 as P
    Wp = PAPER
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    P.build()
    L, T, B = Wp["L"], Wp["T"], Wp["sets"]
    g = torch.Generator(device=dev)
    g.manual_seed(1512)
    cg = P.CG(tol=1e-10, maxit=50000, prec="mixed", delta=args.delta)

    def draw(n, N):
        p = torch.randn((N, 2), generator=g, device=dev, dtype=torch.float64)
        e = torch.view_as_complex(torch.randn((N, 2, 2), generator=g, device=dev,
                                              dtype=torch.float64) * math.sqrt(0.5)).contiguous()
        u = torch.rand(n, generator=g, device=dev, dtype=torch.float64).cpu().numpy()
        return p, e, u

    # thermalisation: 8 chains from the ordered start, 50 trajectories
    # accepted unconditionally, then Metropolis; chain 0 is the configuration
    # (the paper's thermalised configuration is not available)
    t0 = time.time()
    nth = 8
    th = P.Lattice([L] * nth, [T] * nth, Wp["beta"], Wp["m0"], device=dev)
    q = torch.zeros((nth * L * T, 2), dtype=torch.float64, device=dev)
    mdt = P.MD(scheme="adapted_nested_fg", tau=Wp["tau"], n=40, M=Wp["M"], cg=cg)
    acc_th = []
    for k in range(args.therm_paper):
        p, e, u = draw(nth, nth * L * T)
        _, _, a = th.hmc_trajectory(q, p, e, u if k >= 50 else np.zeros(nth), mdt, check=False)
        if k >= 50:
            acc_th.append(a)
    q0 = q[:L * T].clone()
    del th, q
    log(f"paper: thermalised in {time.time() - t0:.1f}s")

    lat = P.Lattice([L] * B, [T] * B, Wp["beta"], Wp["m0"], device=dev)
    qb = q0.repeat(B, 1)

    def measure(scheme, fg, h, merge=True):
        n = int(math.ceil(Wp["tau"] / h - 1e-9))
        md = P.MD(scheme=scheme, tau=Wp["tau"], n=n, M=Wp["M"], fg=fg, cg=cg, tol_action=1e-12,
                  merge_kicks=merge)
        p, e, u = draw(B, B * L * T)
        q = qb.clone()
        dH, _, acc = lat.hmc_trajectory(q, p, e, u, md, check=False)
        st = lat.stats.as_dict()  # this call's counters
        # a trajectory whose |Delta H| exceeds 10 has left the integrator's
        # stability region (it is rejected with probability > 0.99995); its
        # |Delta H| (up to 1e15 here) would swamp the mean of the others
        ok = np.isfinite(dH)
        a = np.abs(dH[ok])
        stable = a[a <= 10.0]
        return {"scheme": scheme, "fg": fg, "h": round(Wp["tau"] / n, 6), "n": n,
                "M": Wp["M"] if "nested" in scheme else None,
                "acceptance": round(float(np.mean(acc)), 4),
                "acceptance_expected": round(float(np.mean(np.exp(np.minimum(0.0, -dH[ok])))), 4),
                "median_abs_dH": float(np.median(a)),
                "mean_abs_dH_stable": float(stable.mean()) if len(stable) else None,
                "err_abs_dH_stable":
                    float(stable.std() / math.sqrt(len(stable))) if len(stable) else None,
                "unstable": int((a > 10.0).sum() + (~ok).sum()),
                "mean_abs_dH_all": float(a.mean()),
                "inversions_per_traj_md": int(st["inversions"])}

    def measure_n(scheme, fg, n, draws, M=Wp["M"], M2=1):
        """Acceptance and inversions at n steps on fixed draws (the same
        momenta and noise for every n of one integrator); the CG iterations
        of the trajectory (all its solves, H included) per chain are its
        cost."""
        md = P.MD(scheme=scheme, tau=Wp["tau"], n=n, M=M, M2=M2, fg=fg, cg=cg, tol_action=1e-12,
                  merge_kicks=False)
        p, e, u = draws
        q = qb.clone()
        dH, _, acc = lat.hmc_trajectory(q, p, e, u, md, check=False)
        st = lat.stats.as_dict()
        ok = np.isfinite(dH)
        return {"n": n, "h": round(Wp["tau"] / n, 6), "acceptance": float(np.mean(acc)),
                "acceptance_expected": float(np.mean(np.exp(np.minimum(0.0, -dH[ok]))) * ok.mean()),
                "inversions_per_traj_md": int(st["inversions"]),
                "cg_iterations_per_traj": round(st["chain_iterations"] / B, 1)}

    def h_at_90(scheme, fg, h_paper, M=Wp["M"], M2=1):
        """The step size at 90 % acceptance: the smallest n = tau / h whose
        expected acceptance <min(1, e^-dH)> over the 200 momentum sets is at
        least 0.9, found by bracketing from the paper's h and bisecting over
        integer n on one fixed set of draws; h90 interpolated linearly in h
        between the bracketing n."""
        draws = draw(B, B * L * T)
        if scheme in ("nested3_leapfrog", "adapted_nested3_fg"):
            p3, e3, u3 = draws
            _, e_h, _ = draw(B, B * L * T)
            draws = (p3, torch.cat([e3, e_h]), u3)
        seen = {}

        def A(n):
            if n not in seen:
                seen[n] = measure_n(scheme, fg, n, draws, M, M2)
            return seen[n]["acceptance_expected"]

        n0 = max(2, int(math.ceil(Wp["tau"] / h_paper - 1e-9)))
        if A(n0) >= 0.9:
            hi, lo = n0, max(1, n0 // 2)
            while lo > 1 and A(lo) >= 0.9:
                hi, lo = lo, max(1, lo // 2)
            if A(lo) >= 0.9:
                hi = lo
        else:
            lo, hi = n0, 2 * n0
            while A(hi) < 0.9 and hi < 4096:
                lo, hi = hi, 2 * hi
        while hi - lo > 1:
            mid = (lo + hi) // 2
            if A(mid) >= 0.9:
                hi = mid
            else:
                lo = mid
        a_hi, h_hi = A(hi), Wp["tau"] / hi
        h90 = h_hi
        if lo != hi:
            a_lo, h_lo = A(lo), Wp["tau"] / lo
            if a_lo < 0.9 <= a_hi and a_hi > a_lo:
                h90 = h_lo + (0.9 - a_lo) * (h_hi - h_lo) / (a_hi - a_lo)
        r = seen[hi]
        return {"h90": round(h90, 5), "n": hi, "h_at_n": round(h_hi, 6),
                "acceptance_expected_at_n": round(a_hi, 4),
                "acceptance_at_n": round(r["acceptance"], 4),
                "inversions_per_traj_md_at_n": r["inversions_per_traj_md"],
                "cg_iterations_per_traj_at_n": r["cg_iterations_per_traj"],
                "evaluated": sorted(({"n": k, "acceptance_expected": round(v["acceptance_expected"], 4)}
                                     for k, v in seen.items()), key=lambda d: d["n"])}

    t1 = time.time()
    table = []
    for scheme, fg, h, per_step, per_traj in Wp["table1"]:
        # the paper counts every kick of every step; adjacent kicks of the
        # same force merged into one (same flow) need fewer inversions
        r = measure(scheme, fg, h, merge=False)
        r["inversions_per_traj_md_merged_kicks"] = measure(scheme, fg, h)["inversions_per_traj_md"]
        r.update({"paper_h": h, "paper_inversions_per_step": per_step,
                  "paper_inversions_per_traj": per_traj})
        if not args.no_h90:
            r["at_90_percent"] = h_at_90(scheme, fg, h)
            log(f"paper h90 {scheme}/{fg}: {r['at_90_percent']}")
        table.append(r)
        log(f"paper table1 {scheme}/{fg} h={r['h']}: acc {r['acceptance']} median |dH| "
            f"{r['median_abs_dH']:.4g} unstable {r['unstable']} inversions "
            f"{r['inversions_per_traj_md']}")
    # the outlook of the paper's Conclusions: the determinant split over two
    # masses, three time scales, the force-gradient term for the ratio part
    # only; each variant at its own 90 % step size, its cost in CG iterations
    # per trajectory beside the two-level adapted scheme's
    three = None
    if not args.no_h90 and not args.no_three_level:
        base = next(r["at_90_percent"] for r in table if r["scheme"] == "adapted_nested_fg")
        three = {"two_level_adapted_nested_fg": {
            "h90": base["h90"], "n": base["n"],
            "cg_iterations_per_traj": base["cg_iterations_per_traj_at_n"],
            "inversions_per_traj_md": base["inversions_per_traj_md_at_n"]}, "variants": []}
        for dm in Wp["heavy_dm"]:
            lat.set_heavy(dm)
            for M2 in Wp["M2"]:
                M = max(1, int(math.ceil(Wp["M"] / M2)))  # the gauge micro step ~ h/10
                r = h_at_90("adapted_nested3_fg", "exact", 0.056, M=M, M2=M2)
                r.update({"dm": dm, "M2": M2, "M": M})
                three["variants"].append(r)
                log(f"paper three-level dm={dm} M2={M2} M={M}: h90 {r['h90']} cg iters/traj "
                    f"{r['cg_iterations_per_traj_at_n']} (two-level "
                    f"{base['cg_iterations_per_traj_at_n']})")
    scan = []
    for scheme, fg in Wp["scan"]:
        for h in Wp["scan_h"]:
            scan.append(measure(scheme, fg, h))
    dt = time.time() - t1
    ntraj = B * (len(table) + len(scan) + sum(len(r.get("at_90_percent", {}).get("evaluated", []))
                                             for r in table)
                 + (sum(len(v["evaluated"]) for v in three["variants"]) if three else 0))
    res = {
        "metric": "paper workload: trajectories/s over the Table 1 and Fig. 1 runs",
        "value": round(ntraj / dt, 3), "unit": "trajectories/s", "n_gpus": 1,
        "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic (own thermalised start)",
        "config": {"workload": "32x32 beta=1.0 m0=-0.231367 tau=2, 200 momentum sets per "
                               "integrator and step size, nested micro step h/10 (M=5), mixed "
                               "CG tol 1e-10 (1e-12 for the S_F of H)",
                   "thermalisation": {"chains": nth, "trajectories": args.therm_paper,
                                      "acceptance_after_50":
                                          round(float(np.mean(np.concatenate(acc_th))), 4)
                                          if acc_th else None}},
        "inversions_counting": "D^-1 per trajectory in the MD (one D^dag D solve = 2; the "
                               "two solves of H are not counted); Table 1 rows with every kick "
                               "evaluated (as the paper counts), plus the merged-kick count",
        "table1": table, "scan": scan, "three_level": three}
    if args.out:
        with open(args.out, "w") as f:
            f.write(json.dumps(res, indent=1) + "\n")
    print(json.dumps(res), flush=True)


# ------------------------------------------------- D^dag D at 2048 x 2048 --

DDAGD_FLOPS_PER_SITE = 112  # two stages of 4 hops x 11 flops + 12 for the diagonal


def measure_ddagd(torch, P, dev, reps=20, prec="f32", warmup=3, rates=None):
    """Fused D^dag D (sm_apply_DdagD) on one 2048 x 2048 lattice; algorithmic
    bytes 48 (FP32) or 96 (FP64) per site: read in and U once, write out once.

    The headline figure times `reps` launches back to back inside one event
    pair, alternating between two independent sets of (U, in, out), so that
    no launch finds its operands in L2 and each pays for the write-back of
    its predecessor's output: in steady state a launch's DRAM traffic is its
    algorithmic bytes.  The single-launch figure (L2 flushed and clean before
    each launch, one event pair per launch) is kept beside it: it does not
    pay for its own output still dirty in L2 when the kernel ends."""
    L = T = 2048
    lat = P.Lattice(L, T, 8.0, kappa_to_m0(0.255), device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    cdt = torch.complex64 if prec == "f32" else torch.complex128
    sets = []
    for _ in range(2):
        q = (torch.rand((L * T, 2), generator=g, device=dev, dtype=torch.float64) * 2 - 1) * math.pi
        U64, U32 = lat.links(q)
        psi = torch.randn((L * T, 2), generator=g, device=dev, dtype=cdt)
        sets.append((U32 if prec == "f32" else U64, psi, torch.empty_like(psi)))
        del q
    # L2 flush: write 256 MiB (evicts the operands), then read another 256
    # MiB, so that the flush's own dirty lines are written back before the
    # timed launch instead of inside it
    flush = torch.empty(int(256 * 2 ** 20), dtype=torch.uint8, device=dev)
    clean = torch.zeros(int(32 * 2 ** 20), dtype=torch.int64, device=dev)
    tuned = None
    if prec == "f32":
        # the streaming form's strip height, picked by the library's autotuner
        h, cand = lat.autotune_ddagd(*sets[0])
        tuned = {"strip_height": h, "candidates_ms": [[a, round(b, 4)] for a, b in cand]}
    for i in range(warmup):
        U, psi, out = sets[i % 2]
        lat.apply_DdagD(U, psi, out)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # back to back, from a clean L2: blocks of `per` launches, the median
    # block
    per = max(reps, 40)
    blocks = []
    for _ in range(5):
        flush.fill_(2)
        clean.sum()
        torch.cuda.synchronize()
        e0.record()
        for i in range(per):
            U, psi, out = sets[i % 2]
            lat.apply_DdagD(U, psi, out)
        e1.record()
        torch.cuda.synchronize()
        blocks.append(e0.elapsed_time(e1) / per)
    ms_b2b = float(np.median(blocks))
    # one launch per event pair
    ts = []
    for i in range(reps):
        U, psi, out = sets[i % 2]
        flush.fill_(2)
        clean.sum()
        e0.record()
        lat.apply_DdagD(U, psi, out)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.median(ts))
    bps = 48 if prec == "f32" else 96
    gbs = bps * L * T / (ms_b2b / 1e3) / 1e9
    gbs1 = bps * L * T / (ms / 1e3) / 1e9
    peaks, src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    kname = "k_ddagd_stream" if prec == "f32" else "k_ddagd_tile<double>"
    return {"kernel": kname, "lattice": "2048x2048",
            "ms_per_launch": round(ms_b2b, 4), "bytes_per_site": bps,
            "algorithmic_bytes_per_launch": bps * L * T, "achieved": round(gbs, 1),
            "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 4), "peak_source": src,
            "timing": f"{per} launches back to back per event pair (median of 5 such blocks), "
                      "two alternating operand sets (402 MB), L2 clean at the start of a block",
            "ms_per_launch_blocks": [round(b, 4) for b in blocks],
            "single_launch": {"ms_median": round(ms, 4), "achieved": round(gbs1, 1),
                              "frac": round(gbs1 / hbm, 4),
                              "l2": "flushed and clean before each launch (write 256 MiB, then "
                                    "read 256 MiB); the launch's own dirty output is written "
                                    "back after its end event"},
            "reps": reps, "autotune": tuned,
            "traffic": ncu_traffic(kname) if prec == "f32" else None,
            "traffic_unit": "DRAM bytes per launch (ncu, back-to-back launches, cache control "
                            "none)",
            **fp64_roofline(ms_b2b, L * T, prec, rates)}


def fp64_roofline(ms, sites, prec, rates):
    """The FP64 stencil against the measured FP64 FMA rate (its bound on
    GB300: 112 flops per 96 bytes needs ~7.8 TFLOP/s to keep up with HBM)."""
    if prec != "f64" or not rates:
        return {}
    tf = DDAGD_FLOPS_PER_SITE * sites / (ms / 1e3) / 1e12
    return {"alu": {"bound": "fp64", "flops_per_site": DDAGD_FLOPS_PER_SITE,
                    "achieved_tflops": round(tf, 4),
                    "peak_tflops": round(rates["fp64_tflops"], 4),
                    "frac": round(tf / rates["fp64_tflops"], 4),
                    "peak_source": "measured in this run (sm_peak_fma, FP64)"}}


# ------------------------------------------------------- oracle (CPU) ------

def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _oracle_trajectory(job):
    """One HMC trajectory of one 64 x 64 chain of the workload with the FP64
    oracle (a worker of the CPU baseline); job = (q, p, eta, u) of the chain,
    host arrays in the site-major layout.  Returns its seconds."""
    from oracle import integrators as ig
    from oracle import schwinger as sw
    W = WORKLOAD
    L, T = W["L"], W["T"]
    q, p, eta, u = job
    lat = sw.Lattice(L, T, W["beta"], kappa_to_m0(W["kappa"]))
    t0 = time.time()
    ig.hmc_trajectory(lat, q.reshape(T, L, 2), p.reshape(T, L, 2), eta.reshape(T, L, 2), u,
                      W["scheme"], W["tau"], W["n"], M=W["M"], fg=W["fg"],
                      solver=sw.Solver(tol=W["cg_tol"]))
    return time.time() - t0


def _noop(x):
    return x


class OraclePool:
    """A process pool of single-threaded oracle workers, one per host core,
    started with `spawn` (a forked copy of a process that holds a CUDA
    context can hang)."""

    def __init__(self, cores):
        import multiprocessing as mp
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"  # inherited by the workers: one thread each
        self.cores = cores
        self.pool = mp.get_context("spawn").Pool(cores)
        self.pool.map(_noop, range(cores))  # workers up before any timing

    def run(self, jobs):
        """Runs the jobs; returns (wall seconds, per-job seconds)."""
        t0 = time.time()
        ts = self.pool.map(_oracle_trajectory, jobs, chunksize=1)
        return time.time() - t0, ts

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(jobs):
    """The oracle timed on the host cores: one trajectory of each of the
    first `cores` chains in parallel (one single-threaded worker per core),
    and one trajectory alone on one core (the 1-thread figure)."""
    cores = min(host_cores(), len(jobs))
    t1 = _oracle_trajectory(jobs[0])
    pool = OraclePool(cores)
    try:
        wall, ts = pool.run(jobs[:cores])
    finally:
        pool.close()
    return {"value": round(cores / wall, 5), "unit": "trajectories/s", "cores": cores,
            "host_cores": host_cores(), "kind": "oracle",
            "single_thread": {"value": round(1.0 / t1, 5), "cores": 1, "seconds": round(t1, 2)},
            "sample": f"1 trajectory of each of {cores} chains (64x64, the GPU arm's thermalised "
                      f"start and its first timed step's momenta, noise and uniforms), one "
                      f"single-threaded numpy FP64 worker per core, {wall:.1f}s wall "
                      f"(mean {np.mean(ts):.1f}s per trajectory)"}


def oracle_start(seed=99, ntraj=20):
    """A start configuration for the reference arm thermalised by the oracle
    alone: the first phase of the GPU arm's thermalisation (heavy fermions,
    kappa = 0.10, nested leapfrog n = 5, M = 8, every trajectory accepted),
    cheap on the host because its solves converge in a few dozen
    iterations."""
    from oracle import integrators as ig
    from oracle import schwinger as sw
    from paper_1512_03812_gb300 import inputs as I
    W = WORKLOAD
    L, T = W["L"], W["T"]
    lat = sw.Lattice(L, T, W["beta"], kappa_to_m0(0.10))
    q = np.zeros((T, L, 2))
    for k in range(ntraj):
        r = ig.hmc_trajectory(lat, q, I.momenta(L, T, seed + 2 * k).reshape(T, L, 2),
                              I.noise(L, T, seed + 2 * k + 1).reshape(T, L, 2), 0.0,
                              "nested_leapfrog", 1.0, 5, M=8, solver=sw.Solver(tol=1e-8))
        q = r.q_md
    return q.reshape(L * T, 2)


def run_reference(args):
    """The oracle as the reference arm: each step one trajectory of each of
    `cores` chains in parallel on the host cores (a bounded sample of the
    workload; rank 0 only)."""
    world, rank, _ = rank_env()
    if rank != 0:
        return
    from paper_1512_03812_gb300 import inputs as I
    W = WORKLOAD
    L, T = W["L"], W["T"]
    t0 = time.time()
    q = oracle_start()
    log(f"reference: oracle start thermalised in {time.time() - t0:.1f}s")
    cores = host_cores()
    pool = OraclePool(cores)

    def jobs(step):
        s = 1000 + 97 * step
        return [(q, I.momenta(L, T, s + 3 * c), I.noise(L, T, s + 3 * c + 1),
                 float(I.uniforms(1, s + 3 * c + 2)[0])) for c in range(cores)]

    try:
        for i in range(args.warmup):
            pool.run(jobs(i))
        walls = [pool.run(jobs(args.warmup + i))[0] for i in range(args.steps)]
    finally:
        pool.close()
    v = args.steps * cores / sum(walls)
    sample = (f"per step 1 trajectory of each of {cores} chains in parallel, one single-threaded "
              f"numpy FP64 worker per host core; start thermalised by the oracle (kappa 0.10)")
    print(json.dumps({
        "impl": "reference", "metric": "HMC trajectories/s", "value": round(v, 5),
        "unit": "trajectories/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * sum(walls) / len(walls), 1), "higher_is_better": True,
        "scaling": "weak", "config": bench_config(W, args.chains, world, args), "dtype": "f64",
        "data": "synthetic (oracle-thermalised start, seeded momenta/noise)",
        "cpu_baseline": {"value": round(v, 5), "unit": "trajectories/s", "kind": "oracle",
                         "cores": cores, "sample": sample},
        "e2e": {"value": round(v, 5), "unit": "trajectories/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)


def run_stencil(args):
    """The fused D^dag D stencil alone on one 2048 x 2048 lattice, FP32 (the
    line's value) and FP64, --steps timed launches each."""
    import torch

    import paper_1512_03812_gb300 as P
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    P.build()
    from paper_1512_03812_gb300 import binding
    rates = binding.measure_peaks()
    f32 = measure_ddagd(torch, P, dev, reps=args.steps, prec="f32", warmup=args.warmup)
    f64 = measure_ddagd(torch, P, dev, reps=args.steps, prec="f64", warmup=args.warmup,
                        rates=rates)
    print(json.dumps({"metric": "fused D^dag D stencil, algorithmic GB/s", "value": f32["achieved"],
                      "unit": "GB/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": f32["ms_per_launch"], "higher_is_better": True,
                      "dtype": "f32", "data": "synthetic (random links and spinor)",
                      "config": {"workload": "D^dag D, 2048x2048 beta=8.0 kappa=0.255",
                                 "l2": f32["timing"]},
                      "roofline": {"bound": "hbm", "achieved": f32["achieved"],
                                   "peak": f32["peak"], "unit": "GB/s", "frac": f32["frac"],
                                   "kernel": f32["kernel"],
                                   "traffic": f32["traffic"],
                                   "traffic_unit": f32["traffic_unit"]},
                      "single_launch": f32["single_launch"], "autotune": f32["autotune"],
                      "f64": f64, "measured_rates": rates}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chains", type=int, default=WORKLOAD["chains_per_gpu"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "f64"])
    ap.add_argument("--therm", type=int, default=20)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--tight-tol", type=float, default=1e-12,
                    help="also time both paths at this CG tolerance and compare Delta H (0: skip)")
    ap.add_argument("--tight-steps", type=int, default=2,
                    help="trajectories per arm of the tight-tolerance comparison")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ddagd", action="store_true")
    ap.add_argument("--cg-variant", type=int, default=-1)
    ap.add_argument("--graph", action="store_true",
                    help="replay one captured trajectory (CUDA graph) per step")
    ap.add_argument("--workload", default="default",
                    choices=["default", "batched", "large", "stencil", "paper", "sweep"])
    ap.add_argument("--out", default=None, help="also write the JSON result to this file")
    ap.add_argument("--therm-paper", type=int, default=150,
                    help="thermalisation trajectories of the paper workload")
    ap.add_argument("--no-three-level", action="store_true",
                    help="paper workload: skip the three-level (determinant split) variants")
    ap.add_argument("--no-h90", action="store_true",
                    help="paper workload: skip the search for the 90 %% acceptance step size")
    ap.add_argument("--n", type=int, default=WORKLOAD["n"])
    ap.add_argument("--M", type=int, default=WORKLOAD["M"])
    ap.add_argument("--delta", type=float, default=None,
                    help="reliable-update factor of the mixed CG (default: the workload's, "
                         "0.0003 for the 64x64 chains, 0.001 for the others)")
    ap.add_argument("--algo", default="auto", choices=["auto", "grid", "chain"])
    ap.add_argument("--sf-start", default="solve", choices=["solve", "noise"],
                    help="S_F in H at the start of a trajectory: a CG solve (default) or "
                         "eta^dag eta, exact for phi = D^dag eta (one solve fewer)")
    ap.add_argument("--rank-selftest", action="store_true",
                    help="run only the rank logic of a multi-rank launch (gloo, no GPU)")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one process per GPU: start the ranks and wait for them
        sys.exit(launch_ranks(args.gpus, sys.argv[1:]).returncode)
    if args.rank_selftest:
        run_rank_selftest(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "stencil":
        run_stencil(args)
    elif args.workload == "sweep":
        if args.delta is None:
            args.delta = WORKLOAD["cg_delta"]
        run_sweep(args)
    elif args.workload == "paper":
        if args.delta is None:
            args.delta = PAPER["cg_delta"]
        run_paper(args)
    elif args.workload != "default":
        if args.delta is None:
            args.delta = OTHER_WORKLOADS[args.workload]["cg_delta"]
        run_other(args)
    else:
        if args.delta is None:
            args.delta = WORKLOAD["cg_delta"]
        run_ours(args)


if __name__ == "__main__":
    main()
