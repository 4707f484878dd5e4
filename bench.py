"""Throughput benchmark of the GB300 central-moment LBM (one JSON line on rank 0).

Default workload: the 256^3 smoke plume (inflow disk of radius 16 at u = 0.1 with a seeded
+/-1 % perturbation, voxelised sphere of radius 24, open faces, nu = 1e-5, passive scalar),
FP32 storage.  A step is one reference step of the whole hot path: one fused
collide-stream + scalar launch over every node.  The state (1.9 GB) is far larger than L2,
so no flush is needed between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload plume256|plume256_fp16]
                  [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle (the reference arm of this build: there is
no runnable reference code) on a bounded sample of the same workload.
Under torchrun each rank advances its own replica (the single-domain workload is not
partitioned: "replicas only"); value = all ranks' lattice updates / max wall time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def _kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1807_02284_gb300", "csrc")
    for fn in ("lbm_device.cuh", "lbm_cell.cuh", "kernels_step.cu"):
        with open(os.path.join(csrc, fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(workload):
    """DRAM bytes per launch of the collide-stream kernel from the committed ncu summary,
    or None when the summary is missing or was taken on different kernel sources."""
    path = os.path.join(ROOT, "profiles", f"k_step_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    hm = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    if not m or not hm or hm.group(1) != _kernel_source_hash():
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"lbm_clocks_{os.getpid()}.csv")
        self.nvml = None

    def _nvml_open(self):
        """Read-only NVML queries through ctypes (no Python NVML package on every host): the
        device with the same UUID as the CUDA device.  None when NVML is not available."""
        import ctypes
        import threading
        import torch
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            uuid = "GPU-" + str(torch.cuda.get_device_properties(self.dev).uuid)
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h)) != 0:
                return None
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) != 0:   # 1: SM clock
                return None
            return {"lib": lib, "h": h, "max": mx.value, "samples": [], "stop": threading.Event()}
        except Exception:
            return None

    def _nvml_loop(self):
        import ctypes
        n = self.nvml
        mhz, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while not n["stop"].is_set():
            if (n["lib"].nvmlDeviceGetClockInfo(n["h"], 1, ctypes.byref(mhz)) == 0 and
                    n["lib"].nvmlDeviceGetCurrentClocksEventReasons(n["h"], ctypes.byref(rs)) == 0):
                n["samples"].append((mhz.value, rs.value))
            n["stop"].wait(0.01)

    def start(self):
        self.nvml = self._nvml_open()
        if self.nvml is not None:
            import threading
            self.thread = threading.Thread(target=self._nvml_loop, daemon=True)
            self.thread.start()
            return
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.nvml is not None:
            self.nvml["stop"].set()
            self.thread.join(timeout=5)
            smp = self.nvml["samples"]
            if not smp:
                return None
            # clock event reason bits: 0x4 sw power cap, 0x8 hw slowdown, 0x20 sw thermal,
            # 0x40 hw thermal
            bits = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown",
                    0x4: "sw_power_cap"}
            reasons = sorted({name for _, r in smp for b, name in bits.items() if r & b})
            return {"sm_mhz": float(np.median([m for m, _ in smp])),
                    "sm_max_mhz": float(self.nvml["max"]), "reasons": reasons,
                    "samples": len(smp), "source": "nvml, every 10 ms"}
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(ws, val):
    if ws == 1:
        return val
    import torch
    import torch.distributed as dist
    t = torch.tensor([val], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def timed_repeats(ws, dev, stream, run_k, reset=None, min_total_s=1.0, min_repeats=3,
                  max_repeats=400):
    """Times repeated calls of ``run_k`` (one call = the K timed steps), each bracketed by a
    barrier and a device synchronize on both sides and timed with CUDA events on the
    library's stream, until at least ``min_total_s`` of device time and ``min_repeats`` calls
    have been taken.  ``reset`` (untimed, before every call after the first) puts the
    workload back to its state before the first call, so every call steps the same flow
    (the scenes are only stable for their configured number of steps).  Clocks are sampled
    across all calls.  Returns the per-call device times (max over ranks) and the clock
    record."""
    import torch
    clocks = ClockSampler(dev)
    times, total = [], 0.0
    clocks.start()
    while len(times) < max_repeats and (len(times) < min_repeats or total < min_total_s):
        if times and reset is not None:
            reset()
            torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        _barrier(ws)
        torch.cuda.synchronize()
        ev0.record(stream)
        run_k()
        ev1.record(stream)
        ev1.synchronize()
        torch.cuda.synchronize()
        _barrier(ws)
        t = _max_over_ranks(ws, ev0.elapsed_time(ev1) / 1e3)
        times.append(t)
        total += t
    clk = clocks.stop()
    return times, clk


def repeat_record(times, K, units_per_step):
    """Summary of the repeated timed calls: the median call gives ``value``."""
    ts = sorted(times)
    med = float(np.median(ts))
    return {"count": len(ts), "steps_per_call": K, "ms_per_step_median": med / K * 1e3,
            "ms_per_step_best": ts[0] / K * 1e3, "ms_per_step_worst": ts[-1] / K * 1e3,
            "value_best": units_per_step * K / ts[0] / 1e6,
            "device_seconds": float(sum(ts))}


def _workload(name):
    import synth
    storage = "fp16" if name.endswith("fp16") else "fp32"
    if name.startswith("multiscale3"):     # also multiscale3_regwall
        return synth.multiscale(scale=1.0), "fp32"
    if name == "farfield256":       # the plume inside a far-field block of spacing 2
        sc = synth.plume(256)
        sc.blocks.append(synth.far_block(sc.blocks[0], 2.0, 64.0, seed=9, amp=0.0))
        return sc, "fp32"
    m = re.match(r"plume(\d+)", name)       # plume256, plume128_fp16, plume256_walls, ...
    sc = synth.plume(int(m.group(1)) if m else 256)
    return sc, storage


def _algorithmic_bytes(flags, storage, local=False):
    """Bytes the collide-stream launch must move per step, by node kind: fluid nodes read
    and write 27 populations, the lagged velocity (not read when the strain rate is taken
    from the node's own moments) and the scalar; obstacle voxels only write their rest state;
    inflow nodes read their velocity and write their equilibrium."""
    pop = 2 if storage == "fp16" else 4
    solid = int(((flags & 1) != 0).sum())
    inflow = int(((flags & 2) != 0).sum()) - int(((flags & 3) == 3).sum())
    fluid = flags.size - solid - inflow
    per_fluid = 27 * pop * 2 + 12 * (1 if local else 2) + 4 * 2 + 1
    per_solid = 27 * pop + 12 + 4 + 1
    per_inflow = 27 * pop + 12 * 2 + 4 * 2 + 1
    return fluid * per_fluid + solid * per_solid + inflow * per_inflow, per_fluid


def _oracle_rate(st, p, budget_s, threads):
    """Steps the oracle (as it stands) with ``threads`` intra-op threads until ``budget_s``
    seconds have passed (at least one step); returns (steps, seconds, state)."""
    import torch

    from oracle import grid
    prev = torch.get_num_threads()
    torch.set_num_threads(threads)
    try:
        n = 0
        t0 = time.perf_counter()
        while True:
            st = grid.step(st, p)
            n += 1
            el = time.perf_counter() - t0
            if el >= budget_s:
                break
    finally:
        torch.set_num_threads(prev)
    return n, el, st


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _outer_layer(dims):
    nx, ny, nz = dims
    m = np.zeros((nz, ny, nx), bool)
    m[0], m[-1], m[:, 0], m[:, -1], m[:, :, 0], m[:, :, -1] = (True,) * 6
    return m


def _positions(blk, mask):
    z, y, x = np.nonzero(mask)
    o = np.asarray(blk.origin, float)
    return np.stack([o[0] + blk.h * x, o[1] + blk.h * y, o[2] + blk.h * z], 1)


def _source_nodes(src, pos):
    """Distinct nodes of block ``src`` that the trilinear interpolation at reference-unit
    points ``pos`` reads with a non-zero weight (obstacle corners dropped), as in the
    mapping kernel."""
    dims = np.asarray(src.dims)
    q = (pos - np.asarray(src.origin, float)) / src.h
    i0 = np.clip(np.floor(q + 1e-9).astype(np.int64), 0, np.maximum(dims - 2, 0))
    t = q - i0
    solid = (src.flags & 1) != 0
    keys = []
    for c in range(8):
        off = np.array([c & 1, (c >> 1) & 1, c >> 2])
        w = np.prod(np.where(off[None, :] == 1, t, 1.0 - t), axis=1)
        idx = np.minimum(i0 + off[None, :], dims[None, :] - 1)
        lin = (idx[:, 2] * dims[1] + idx[:, 1]) * dims[0] + idx[:, 0]
        keep = (w > 1e-12) & ~solid.reshape(-1)[lin]
        keys.append(lin[keep])
    return int(np.unique(np.concatenate(keys)).size)


def _coupling_bytes(sc, subs):
    """Algorithmic bytes per reference step of the continuous-scale coupling (Sec. 3.2,
    4.2.4, 4.2.5) beyond the collide-stream updates: each mapping writes 27 populations,
    the velocity and the scalar of each destination node (124 B) and reads 27 populations,
    the scalar and the flag byte of every distinct source node it interpolates from (113 B
    per source time level); the fused temporal alignment also reads each updated node's
    populations and scalar at t_n (112 B).  A refined block with l sub-steps takes l + 1
    ghost-layer mappings per step (the refresh at t_n, one before each later sub-step, the
    one at t_n + dt_0), reading 2 l source levels in total; post-mapping reads one level."""
    blocks = sc.blocks
    out = {"ghost": 0, "post": 0, "align": 0}
    W, R = 124, 113
    for i, b in enumerate(blocks[1:], start=1):
        if b.h >= 1.0:
            continue
        lo = np.asarray(b.origin, float)
        hi = lo + (np.asarray(b.dims) - 1) * b.h
        par = 0
        for j, c in enumerate(blocks[1:], start=1):      # nearest coarser block around b
            clo = np.asarray(c.origin, float)
            chi = clo + (np.asarray(c.dims) - 1) * c.h
            if j != i and c.h > b.h and np.all(clo <= lo + 1e-9) and np.all(hi <= chi + 1e-9) \
                    and c.h < blocks[par].h:
                par = j
        ghost = _outer_layer(b.dims) & ((b.flags & 1) == 0)
        l = subs[i]
        src = _source_nodes(blocks[par], _positions(b, ghost))
        out["ghost"] += (l + 1) * int(ghost.sum()) * W + 2 * l * src * R
        if abs(1.0 / b.h - round(1.0 / b.h)) > 1e-9:
            upd = (~_outer_layer(b.dims)) & ((b.flags & 1) == 0)
            out["align"] += int(upd.sum()) * 112
        ilo, ihi = lo + b.h, hi - b.h
        interior = np.zeros(b.shape_zyx, bool)
        interior[1:-1, 1:-1, 1:-1] = True
        for k, t in enumerate(blocks):
            if not t.h > b.h:
                continue
            tpos = _positions(t, np.ones(t.shape_zyx, bool))
            inside = np.all((tpos >= ilo - 1e-9) & (tpos <= ihi + 1e-9), axis=1)
            tmask = inside.reshape(t.shape_zyx) & ((t.flags & 1) == 0)
            if k > 0:
                tmask &= ~_outer_layer(t.dims)
            n_t = int(tmask.sum())
            if n_t:
                out["post"] += n_t * W + _source_nodes(b, _positions(t, tmask)) * R
    out["total"] = out["ghost"] + out["post"] + out["align"]
    return out


def cpu_baseline_measure(budget_s=24.0, storage="fp32"):
    """The FP64 oracle as it stands, on a bounded sample of the plume workload: the same
    scene geometry scaled to a 32^3 box (inflow disk, sphere, open faces), timed with one
    thread (a third of ``budget_s``) and with every host core (the rest).  The oracle's cost
    per node and step does not depend on the box size, so the sample's rate is the rate of
    the full workload (labelled as an extrapolation).  The GPU path then runs the same sample
    from the same (float32-rounded) inputs for the same number of steps as the all-core run,
    and the velocity error against the oracle is reported with the timing."""
    import synth
    from oracle import grid
    from paper_1807_02284_gb300 import lbm
    sc = synth.plume(32)
    b = sc.blocks[0]
    r32 = lambda a: np.asarray(a, dtype=np.float32)
    st0 = grid.init_state(r32(b.rho0).astype(np.float64), r32(b.u0).astype(np.float64),
                          r32(b.c0).astype(np.float64), b.flags)
    p = grid.Params(nu=sc.nu, periodic=sc.periodic, adaptive=sc.adaptive, c_src=sc.c_src)
    cores = _host_cores()
    grid.step(st0, p)  # warm-up
    n1, el1, _ = _oracle_rate(st0, p, budget_s / 3.0, 1)
    n, el, st = _oracle_rate(st0, p, budget_s * 2.0 / 3.0, cores)
    mlups = b.flags.size * n / el / 1e6
    mlups1 = b.flags.size * n1 / el1 / 1e6
    full = 256 ** 3 * 1000
    dom = lbm.Domain(b.dims, sc.nu, periodic=sc.periodic, storage=storage,
                     adaptive=sc.adaptive, c_src=sc.c_src)
    dom.set_flags(b.flags)
    dom.init_macro(r32(b.u0), rho=r32(b.rho0), c=r32(b.c0))
    dom.step(n)
    u = dom.read_field(lbm.LBM_FIELD_U, lbm.LBM_F64).reshape(st.u.shape)
    c = dom.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F64).reshape(st.c.shape)
    dom.close()
    uo = st.u.numpy()
    umax = float(np.abs(uo).max())
    return {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"oracle (FP64, dense per-node M and LU solve) on the plume geometry "
                      f"scaled to 32^3: {n} full steps in {el:.1f} s on {cores} threads, "
                      f"{n1} in {el1:.1f} s on 1 thread",
            "single_thread": {"value": mlups1, "unit": "MLUPS", "cores": 1, "steps": n1,
                              "seconds": el1},
            "extrapolation": f"MLUPS of the 32^3 sample taken as the rate of the 256^3 plume "
                             f"(cost per node and step is size-independent): its 1000 steps "
                             f"would take {full / (mlups * 1e6) / 86400:.1f} days on "
                             f"{cores} threads, {full / (mlups1 * 1e6) / 86400:.1f} on one",
            "parity": {"steps": n, "storage": storage,
                       "u_max_abs_err_rel": float(np.abs(u - uo).max()) / umax,
                       "scalar_max_abs_err": float(np.abs(c - st.c.numpy()).max()),
                       "bound_u_rel": 1e-5 if storage == "fp32" else None}}


def parity_by_variant():
    """Error against the FP64 oracle of each variant the default line reports, each on a
    small seeded case of its own kind run through the same kernel instances (a few seconds
    of oracle time each).  Errors are max-abs velocity errors relative to max|u| (gradient:
    relative L2 error), with the bound the parity tests hold them to."""
    import dataclasses

    import torch

    import synth
    from oracle import adjoint as oadj
    from oracle import coupling, grid
    from paper_1807_02284_gb300 import lbm
    r32 = lambda a: np.asarray(a, dtype=np.float32)

    def single(sc, steps, storage="fp32", grad_mode="lagged", walls=None, obstacles=False):
        b = sc.blocks[0]
        dom = lbm.Domain(b.dims, sc.nu, periodic=sc.periodic, storage=storage,
                         adaptive=sc.adaptive, c_src=sc.c_src, grad_mode=grad_mode)
        if walls or obstacles:
            dom.set_walls(walls or (False,) * 6, obstacles=obstacles)
        dom.set_flags(b.flags)
        dom.init_macro(r32(b.u0), rho=r32(b.rho0), c=r32(b.c0))
        dom.step(steps)
        u = dom.read_field(lbm.LBM_FIELD_U, lbm.LBM_F64).reshape((3,) + b.shape_zyx)
        dom.close()
        st = grid.init_state(r32(b.rho0).astype(np.float64), r32(b.u0).astype(np.float64),
                             r32(b.c0).astype(np.float64), b.flags)
        p = grid.Params(nu=sc.nu, periodic=sc.periodic, adaptive=sc.adaptive, c_src=sc.c_src,
                        grad_mode=grad_mode)
        if walls:
            p = dataclasses.replace(p, walls=tuple(walls))
        p = dataclasses.replace(p, obstacle_walls=obstacles)
        for _ in range(steps):
            st = grid.step(st, p)
        uo = st.u.numpy()
        return float(np.abs(u - uo).max() / np.abs(uo).max())

    def multi(sc, steps, far=(), obstacle_walls=False):
        dom = lbm.Domain(sc.blocks[0].dims, sc.nu, periodic=sc.periodic, adaptive=sc.adaptive,
                         c_src=sc.c_src)
        if obstacle_walls:
            dom.set_walls((False,) * 6, obstacles=True)
        for b in sc.blocks[1:]:
            dom.add_scale_block(b.origin, b.h, b.dims)
        for i, b in enumerate(sc.blocks):
            dom.set_flags(b.flags, block=i)
            dom.init_macro(r32(b.u0), rho=r32(b.rho0), c=r32(b.c0), block=i)
        ms = coupling.MultiScale.build(sc, obstacle_walls=obstacle_walls)
        for fb in far:                  # far-field blocks (h > 1) around the scene
            fid = dom.add_scale_block(fb.origin, fb.h, fb.dims)
            dom.set_flags(fb.flags, block=fid)
            dom.init_macro(r32(fb.u0), rho=r32(fb.rho0), c=r32(fb.c0), block=fid)
            ms.add_far_block(fb.origin, fb.h, fb.dims, fb.rho0, fb.u0, fb.c0, fb.flags)
        dom.step(steps)
        for _ in range(steps):
            ms.step()
        err, umax = 0.0, 0.0
        for i, b in enumerate(ms.blocks):
            u = dom.read_field(lbm.LBM_FIELD_U, lbm.LBM_F64, i).reshape(tuple(b.state.u.shape))
            uo = b.state.u.numpy()
            err, umax = max(err, float(np.abs(u - uo).max())), max(umax, float(np.abs(uo).max()))
        dom.close()
        return err / umax

    out = {}
    t0 = time.perf_counter()
    plume = synth.random_scene(dims=(24, 20, 20), seed=21, periodic=(False, False, False),
                               spheres=[(10.0, 10.0, 10.0, 3.0)], inflow=(10, 10, 4.0, 0.1),
                               nu=1e-4)
    out["plume256_fp16"] = {"u_max_abs_err_rel": single(plume, 6, storage="fp16"),
                            "bound": 2e-3, "case": "24x20x20 plume-shaped scene, 6 steps"}
    out["plume256_local"] = {"u_max_abs_err_rel": single(plume, 6, grad_mode="local"),
                             "bound": 1e-5, "case": "24x20x20 plume-shaped scene, 6 steps"}
    out["plume256_walls"] = {"u_max_abs_err_rel": single(plume, 6, walls=(False,) * 4 + (True, True)),
                             "bound": 1e-5,
                             "case": "24x20x20 plume-shaped scene, floor + lid walls, 6 steps"}
    out["plume256_regwall"] = {"u_max_abs_err_rel": single(plume, 6, obstacles=True),
                               "bound": 1e-5,
                               "case": "24x20x20 plume-shaped scene, sphere surface as walls, 6 steps"}
    ms = synth.multiscale(scale=0.25, nu=2e-3, flow_amp=0.06)
    out["multiscale3"] = {"u_max_abs_err_rel": multi(ms, 2), "bound": 1e-5,
                          "case": "the 3-block scene scaled by 1/4 (32^3, 24^3, 16^3), 2 reference steps"}
    out["multiscale3_regwall"] = {"u_max_abs_err_rel": multi(ms, 2, obstacle_walls=True),
                                  "bound": 1e-5,
                                  "case": "the same scene, sphere surfaces as walls in every block"}
    far = synth.random_scene(dims=(20, 18, 16), seed=41, periodic=(False, False, False),
                             spheres=[(11.0, 9.0, 8.0, 2.5)], inflow=(9, 8, 3.0, 0.08), nu=0.004)
    fb = synth.far_block(far.blocks[0], 1.5, 6.0, seed=5, amp=0.03)
    out["farfield256"] = {"u_max_abs_err_rel": multi(far, 3, far=(fb,)), "bound": 1e-5,
                          "case": "20x18x16 scene inside a far block at h = 1.5, 3 reference steps"}
    bs = synth.batch(count=2, seed=41, lo=10, hi=16, nu=2e-3)
    worst = 0.0
    doms = []
    for s2 in bs:
        b = s2.blocks[0]
        d = lbm.Domain(b.dims, s2.nu, periodic=s2.periodic, adaptive=s2.adaptive, c_src=s2.c_src)
        d.set_flags(b.flags)
        d.init_macro(r32(b.u0), rho=r32(b.rho0), c=r32(b.c0))
        doms.append(d)
    lbm.step_batch(doms, 3)
    for d, s2 in zip(doms, bs):
        b = s2.blocks[0]
        st = grid.init_state(r32(b.rho0).astype(np.float64), r32(b.u0).astype(np.float64),
                             r32(b.c0).astype(np.float64), b.flags)
        p = grid.Params(nu=s2.nu, periodic=s2.periodic, adaptive=s2.adaptive, c_src=s2.c_src)
        for _ in range(3):
            st = grid.step(st, p)
        u = d.read_field(lbm.LBM_FIELD_U, lbm.LBM_F64).reshape((3,) + b.shape_zyx)
        uo = st.u.numpy()
        worst = max(worst, float(np.abs(u - uo).max() / np.abs(uo).max()))
        d.close()
    out["batch64"] = {"u_max_abs_err_rel": worst, "bound": 1e-5,
                      "case": "2 simulations (edges 10-16) in one persistent launch, 3 steps"}
    sc, target = synth.adjoint_scene(n=12, seed=5, nu=0.01, amp=0.05)
    b = sc.blocks[0]
    dom = lbm.Domain(b.dims, sc.nu, periodic=sc.periodic, adaptive=sc.adaptive)
    dom.set_flags(b.flags)
    dom.init_macro(r32(b.u0), rho=r32(b.rho0), c=r32(b.c0))
    dom.set_tape(3)
    dom.step(8)
    c = dom.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F64)
    dldc = torch.tensor(c - target.reshape(-1), dtype=torch.float32, device="cuda")
    g = torch.empty(3 * b.flags.size, dtype=torch.float32, device="cuda")
    dom.adjoint_step(8, dldc, g)
    dom.sync()
    dom.close()
    p = grid.Params(nu=sc.nu, periodic=sc.periodic, adaptive=sc.adaptive)
    _, go, _ = oadj.loss_and_grad(r32(b.u0).astype(np.float64), r32(b.rho0).astype(np.float64),
                                  r32(b.c0).astype(np.float64), b.flags, p, 8, target)
    go = go.numpy().reshape(-1)
    gg = g.cpu().numpy().astype(np.float64)
    out["adjoint128"] = {"grad_rel_l2_err": float(np.linalg.norm(gg - go) / np.linalg.norm(go)),
                         "bound": 1e-3, "case": "12^3 smoke control, 8 steps, checkpoint every 3"}
    out["seconds"] = time.perf_counter() - t0
    return out


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    steps = max(1, args.steps)
    warm = max(0, args.warmup)
    import torch

    import synth
    from oracle import grid
    sc = synth.plume(32)
    b = sc.blocks[0]
    st = grid.init_state(b.rho0, b.u0, b.c0, b.flags)
    p = grid.Params(nu=sc.nu, periodic=sc.periodic, adaptive=sc.adaptive, c_src=sc.c_src)
    for _ in range(warm):
        st = grid.step(st, p)
    t0 = time.perf_counter()
    for _ in range(steps):
        st = grid.step(st, p)
    el = time.perf_counter() - t0
    mlups = b.flags.size * steps / el / 1e6
    cores = int(torch.get_num_threads())
    sample = (f"oracle (FP64 CPU, dense per-node M and LU solve) on the plume geometry scaled "
              f"to 32^3 (the 256^3 step takes minutes on the CPU), {steps} timed steps on "
              f"{cores} threads")
    line = {"impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": steps, "warmup": warm,
            "ms_per_step": el / steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "plume32_oracle", "nodes": int(b.flags.size),
                       "stands_in_for": "plume256_fp32 (the same geometry scaled to 32^3)",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    import synth
    from paper_1807_02284_gb300 import lbm

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    sc, storage = _workload(args.workload)
    b = sc.blocks[0]
    stream = torch.cuda.Stream(device=dev)
    dom = lbm.Domain(b.dims, sc.nu, periodic=sc.periodic, storage=storage,
                     adaptive=sc.adaptive, c_src=sc.c_src, stream=stream,
                     grad_mode="local" if args.workload.endswith("_local") else "lagged")
    if args.workload.endswith("_walls"):     # no-slip floor and lid (the second-order wall)
        dom.set_walls((False, False, False, False, True, True))
    if args.workload.endswith("_regwall"):   # the sphere's surface as the second-order wall
        dom.set_walls((False,) * 6, obstacles=True)
    for blk in sc.blocks[1:]:
        dom.add_scale_block(blk.origin, blk.h, blk.dims)
    for i, blk in enumerate(sc.blocks):
        dom.set_flags(blk.flags, block=i)

    def init_state():
        for i, blk in enumerate(sc.blocks):
            dom.init_macro(blk.u0.astype(np.float32), rho=blk.rho0.astype(np.float32),
                           c=blk.c0.astype(np.float32), block=i)
    init_state()
    # lattice updates and launches per reference step (refined blocks sub-cycle)
    subs = [dom.info(i).substeps for i in range(len(sc.blocks))]
    N = sum(s * blk.flags.size for s, blk in zip(subs, sc.blocks))
    launches_per_step = 1
    for i in range(1, len(sc.blocks)):
        h = sc.blocks[i].h
        if h > 1.0:                   # far field: aligned step, overlap and boundary maps
            launches_per_step += 3
            continue
        # ghost layer at t_n, the first sub-step, the gather-and-blend ghost layer after it,
        # then a ghost layer and a sub-step per later sub-step; post-maps into i coarser blocks
        launches_per_step += 2 * subs[i] + 1 + i
    K, W = args.steps, args.warmup
    if len(sc.blocks) > 1:
        # multi-block steps replay CUDA graphs captured per level-rotation state: time a
        # whole number of 48-step chunks (a multiple of every rotation period here) after a
        # warm-up of the same length, so the timed call replays the graphs the warm-up captured
        K = max(48, int(round(K / 48.0)) * 48)
        W = max(W, K)

    # ---- device-resident throughput (value) and the collide-stream roofline: the K-step
    # call is repeated until at least a second of device time; value is the median call
    dom.step(W)
    dom.sync()

    def reset():
        init_state()
        dom.step(W)
    times, clk = timed_repeats(ws, dev, stream, lambda: dom.step(K), reset)
    dom.sync()
    t_max = float(np.median(times))
    t_dev = t_max
    value = N * K * ws / t_max / 1e6
    reps = repeat_record(times, K, N * ws)

    alg_bytes, per_fluid = 0, 0
    refined = [blk.h < 1.0 for blk in sc.blocks]
    for i, (s, blk) in enumerate(zip(subs, sc.blocks)):
        fl = blk.flags
        if refined[i]:           # scale-boundary nodes are written by mapping, not updated
            fl = fl[~_outer_layer(blk.dims)]
        ab, per_fluid = _algorithmic_bytes(fl, storage, local=args.workload.endswith("_local"))
        alg_bytes += s * ab
    step_bytes = alg_bytes
    coupling = _coupling_bytes(sc, subs) if any(refined) else None
    if coupling is not None:
        alg_bytes += coupling["total"]
    peak, peak_src = _peaks()
    achieved = alg_bytes / (t_dev / K) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": _profiled_traffic(args.workload),
                "peak_source": peak_src, "kernel": "k_step (fused pull/collide/scalar)",
                "bytes_per_fluid_node": per_fluid}
    if coupling is not None:
        roofline["kernel"] = ("whole Algorithm 1 step: k_step sub-steps (fused alignment) and "
                              "k_map prior- / post-mappings")
        roofline["bytes_per_reference_step"] = {"collide_stream": int(step_bytes),
                                                "alignment": coupling["align"],
                                                "ghost_mappings": coupling["ghost"],
                                                "post_mappings": coupling["post"]}
        roofline["frac_collide_stream_bytes_only"] = step_bytes / (t_dev / K) / 1e9 / peak
    i0 = dom.info(0)
    roofline["launch"] = {"tile": [int(i0.tile[0]), int(i0.tile[1])],
                          "ctas_per_sm": int(i0.ctas_per_sm),
                          "nodes_per_thread": int(i0.nodes_per_thread)}

    # ---- end to end through the public API with host buffers
    E = max(3, min(K, 50))
    recs = synth.inflow_records(b)
    rng = np.random.default_rng(123)
    pinned = torch.empty(recs.nbytes, dtype=torch.uint8, pin_memory=True)
    host_recs = pinned.numpy().view(lbm.INFLOW_RECORD)
    base = np.stack([recs["ux"], recs["uy"], recs["uz"]]).astype(np.float32)
    outs = torch.zeros((E, 5), dtype=torch.float64, pin_memory=True)

    def new_inflow():
        host_recs[:] = recs
        jitter = (1.0 + 0.01 * (2 * rng.random(base.shape) - 1)).astype(np.float32)
        host_recs["ux"] = base[0] * jitter[0]

    # pipelined: step i (its inflow upload and its diagnostics' read-back included) is queued
    # before the diagnostics of step i - 1 are waited for and read
    _barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tickets = []
    for i in range(E):
        new_inflow()
        dom.set_inflow(host_recs)
        tickets.append(dom.step_reduce_async(1, outs[i]))   # the step's own kernel sums them
        if i:
            dom.wait_results(tickets[i - 1])
            red = outs[i - 1].numpy()
    dom.wait_results(tickets[-1])
    red = outs[E - 1].numpy()
    t_e2e = time.perf_counter() - t0
    t_e2e = _max_over_ranks(ws, t_e2e)
    # the same with the blocking call: every step waits for its own diagnostics
    _barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(E):
        new_inflow()
        dom.set_inflow(host_recs)
        red = dom.step_reduce(1)
    t_sync = _max_over_ranks(ws, time.perf_counter() - t0)
    e2e = {"value": N * E * ws / t_e2e / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": int(recs.nbytes), "d2h_bytes_per_step": 5 * 8,
           "steps": E, "api": "per step: lbm_set_boundary(INFLOW, pinned host) + "
                             "lbm_step_reduce_async(1, pinned host); step i's diagnostics "
                             "read (lbm_wait_results) once step i + 1 is queued",
           "blocking_value": N * E * ws / t_sync / 1e6,
           "blocking_api": "per step: lbm_set_boundary(INFLOW) + lbm_step_reduce(1, host)"}

    if rank == 0:
        line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": K,
                "warmup": W, "ms_per_step": t_max / K * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f16-storage/f32-math" if storage == "fp16" else "f32",
                "data": "synthetic",
                "config": {"workload": args.workload if "_" in args.workload
                           else f"{args.workload}_{storage}",
                           "lattice_updates_per_step": int(N),
                           "blocks": [{"dims": list(blk.dims), "h": blk.h, "substeps": s}
                                      for blk, s in zip(sc.blocks, subs)],
                           "storage": storage,
                           "parallelism": "replicas" if ws > 1 else "single",
                           "l2": "inputs larger than L2 (state %.2f GB)" %
                                 (N * (27 * (2 if storage == 'fp16' else 4) * 2 + 32) / 1e9)},
                "gb_per_s_algorithmic": achieved,
                "roofline": roofline,
                "repeats": reps,
                "e2e": e2e,
                "gpu_launches": K * launches_per_step,
                "clocks": clk,
                "mass_check": float(red[0])}
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_measure(args.cpu_budget, storage)
        if ws == 1 and args.workload == "plume256" and not args.no_variants:
            line["variants"] = _variants(args)
            if "cpu_baseline" in line:   # the variants' errors against the FP64 oracle
                try:
                    line["cpu_baseline"]["parity_by_variant"] = parity_by_variant()
                except Exception as ex:  # report, do not hide
                    line["cpu_baseline"]["parity_by_variant"] = {"error": f"{type(ex).__name__}: {ex}"}
        print(json.dumps(line), flush=True)
    dom.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_batch(args):
    """64 independent plumes of uneven size (edges 24..96) advanced by lbm_step_batch: one
    graph-captured persistent launch for all K steps."""
    import torch

    import synth
    from paper_1807_02284_gb300 import lbm

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_1807_02284_gb300 import sharding
    scenes = synth.batch(64, seed=4)
    # independent simulations: largest-first placement by node count, no collective
    mine = [scenes[i] for i in
            sharding.rank_share([s.blocks[0].flags.size for s in scenes], rank, ws)]
    stream = torch.cuda.Stream(device=dev)
    doms = []
    for sc in mine:
        b = sc.blocks[0]
        d = lbm.Domain(b.dims, sc.nu, periodic=sc.periodic, stream=stream)
        d.set_flags(b.flags)
        d.init_macro(b.u0.astype(np.float32), rho=b.rho0.astype(np.float32),
                     c=b.c0.astype(np.float32))
        doms.append(d)
    N = sum(sc.blocks[0].flags.size for sc in mine)
    K, W = args.steps, args.warmup
    lbm.step_batch(doms, W)
    lbm.step_batch(doms, K)          # builds and captures the K-step plan outside the timing
    for d in doms:
        d.sync()
    def reset():
        for sc, d in zip(mine, doms):
            b = sc.blocks[0]
            d.init_macro(b.u0.astype(np.float32), rho=b.rho0.astype(np.float32),
                         c=b.c0.astype(np.float32))
        lbm.step_batch(doms, W)
    times, clk = timed_repeats(ws, dev, stream, lambda: lbm.step_batch(doms, K), reset)
    for d in doms:
        d.sync()
    t_max = float(np.median(times))
    t_dev = t_max
    value = N * K * ws / t_max / 1e6
    reps = repeat_record(times, K, N * ws)
    alg = sum(_algorithmic_bytes(sc.blocks[0].flags, "fp32")[0] for sc in mine)
    peak, peak_src = _peaks()
    achieved = alg / (t_dev / K) / 1e9
    # end to end: per step, every member's inflow update from pinned host, one batched step,
    # and every member's diagnostics read back
    E = max(3, min(K, 20))
    recs = [synth.inflow_records(sc.blocks[0]) for sc in mine]
    pins = []
    for r in recs:
        t = torch.empty(max(1, r.nbytes), dtype=torch.uint8, pin_memory=True)
        a = t.numpy()[: r.nbytes].view(lbm.INFLOW_RECORD)
        a[:] = r
        pins.append((t, a))
    for _ in range(2):               # capture the one-step plans of both level parities
        lbm.step_batch_reduce(doms, 1)
    bouts = torch.zeros((E, len(mine), 5), dtype=torch.float64, pin_memory=True)
    # pipelined: step i queued before the diagnostics of step i - 1 are waited for and read
    _barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tickets = []
    for i in range(E):
        lbm.set_inflow_batch(doms, [a for _, a in pins])
        tickets.append(lbm.step_batch_reduce_async(doms, 1, bouts[i]))   # the step's kernel sums them
        if i:
            doms[0].wait_results(tickets[i - 1])
            red = bouts[i - 1].numpy()
    doms[0].wait_results(tickets[-1])
    t_e2e = _max_over_ranks(ws, time.perf_counter() - t0)
    _barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(E):
        lbm.set_inflow_batch(doms, [a for _, a in pins])
        lbm.step_batch_reduce(doms, 1)
    t_sync = _max_over_ranks(ws, time.perf_counter() - t0)
    if rank == 0:
        line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": K,
                "warmup": W, "ms_per_step": t_max / K * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "batch64_fp32", "simulations": len(scenes),
                           "lattice_updates_per_step": int(N * ws),
                           "parallelism": f"simulations sharded over {ws} ranks" if ws > 1
                           else "single",
                           "l2": "inputs larger than L2 (state %.2f GB)" % (N * 280 / 1e9)},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                             "kernel": "k_batch (persistent, cooperative)"},
                "repeats": reps,
                "e2e": {"value": N * E * ws / t_e2e / 1e6, "unit": "MLUPS",
                        "h2d_bytes_per_step": int(sum(r.nbytes for r in recs)),
                        "d2h_bytes_per_step": 40 * len(mine), "steps": E,
                        "api": "per step: lbm_set_inflow_batch(pinned host) + "
                               "lbm_step_batch_reduce_async(1, pinned host); step i's "
                               "diagnostics read (lbm_wait_results) once step i + 1 is queued",
                        "blocking_value": N * E * ws / t_sync / 1e6,
                        "blocking_api": "per step: lbm_set_inflow_batch + "
                                        "lbm_step_batch_reduce(1, host)"},
                "gpu_launches": 1, "clocks": clk}
        print(json.dumps(line), flush=True)
    for d in doms:
        d.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_adjoint(args, emit=True):
    """Smoke control at 128^3 (periodic, nu = 1e-3): forward K steps recording a checkpoint
    every 20 steps, then the hand-written reverse sweep (recompute + adjoint) back to dL/du0.
    value = lattice updates of the reverse sweep per second."""
    import torch

    import synth
    from paper_1807_02284_gb300 import lbm

    torch.cuda.set_device(0)
    n_edge = 64 if args.workload == "adjoint64" else 128
    sc, target = synth.adjoint_scene(n=n_edge, seed=5, nu=1e-3, amp=0.05, steps=args.steps)
    b = sc.blocks[0]
    stream = torch.cuda.Stream()
    dom = lbm.Domain(b.dims, sc.nu, periodic=sc.periodic, stream=stream)
    dom.set_flags(b.flags)
    N = b.flags.size
    K = args.steps
    u0 = torch.tensor(b.u0.astype(np.float32), device="cuda")
    rho0 = torch.tensor(b.rho0.astype(np.float32), device="cuda")
    c0 = torch.tensor(b.c0.astype(np.float32), device="cuda")
    tgt = torch.tensor(target.astype(np.float32).reshape(-1), device="cuda")
    g = torch.empty(3 * N, dtype=torch.float32, device="cuda")
    c = torch.empty(N, dtype=torch.float32, device="cuda")

    def run_once():
        dom.init_macro(u0, rho=rho0, c=c0)
        dom.set_tape(20)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dom.step(K)
        e1.record(stream)
        dom.read_field(lbm.LBM_FIELD_SCALAR, lbm.LBM_F32, out=c)
        with torch.cuda.stream(stream):
            dldc = (c - tgt).contiguous()
        e3 = torch.cuda.Event(enable_timing=True)
        e3.record(stream)
        dom.adjoint_step(K, dldc, g)
        e2.record(stream)
        e2.synchronize()
        return e0.elapsed_time(e1) / 1e3, e3.elapsed_time(e2) / 1e3

    run_once()                                   # warm-up (allocates tape and buffers)
    clocks = ClockSampler(0)
    clocks.start()
    runs = [run_once() for _ in range(3)]        # median of three forward + reverse runs
    clk = clocks.stop()
    t_fwd = float(np.median([r[0] for r in runs]))
    t_rev = float(np.median([r[1] for r in runs]))
    dom.sync()
    peak, peak_src = _peaks()
    # reverse step per fluid node: pass A 393 B (pulled f, Lam in/out, lagged u, adjoints of
    # u and c, scalar, mu out), pass B 69 B, recompute 249 B
    per_node = 393 + 69 + 249
    achieved = N * K * per_node / t_rev / 1e9
    out = {"metric": "MLUPS", "value": N * K / t_rev / 1e6, "unit": "MLUPS",
           "what": "reverse sweep (segment recompute + adjoint) lattice updates per second",
           "forward_with_tape_mlups": N * K / t_fwd / 1e6, "steps": K,
           "config": {"workload": f"adjoint{n_edge}_fp32", "nodes": int(N), "checkpoint_every": 20},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                        "bytes_per_reverse_update": per_node},
           "repeats": {"count": len(runs), "reverse_s": [r[1] for r in runs],
                       "forward_s": [r[0] for r in runs]},
           "gradient_norm": float(torch.linalg.norm(g)), "clocks": clk}
    dom.close()
    if emit:
        print(json.dumps(out), flush=True)
    return out


def run_dynamic(args, emit=True):
    """256^3 plume with a dynamic scale (Sec. 5) at h = 1/2 over the developed jet, rebuilt
    every 40 steps from the gradient and velocity thresholds.  value = lattice updates of all
    blocks per second (sub-cycled updates counted), rebuilds (detection, removal, placement,
    start from the coarse scale, graph re-capture) included in the timed region."""
    import torch

    from paper_1807_02284_gb300 import lbm

    torch.cuda.set_device(0)
    sc, _ = _workload("plume256")
    b = sc.blocks[0]
    stream = torch.cuda.Stream()
    dom = lbm.Domain(b.dims, sc.nu, periodic=sc.periodic, adaptive=sc.adaptive,
                     c_src=sc.c_src, stream=stream)
    dom.set_flags(b.flags)
    dom.init_macro(b.u0.astype(np.float32), rho=b.rho0.astype(np.float32),
                   c=b.c0.astype(np.float32))
    N0 = b.flags.size
    dom.step(400)                                  # develop the jet before tracking it
    u_thr, g_thr = 0.05, 0.02                      # |u| above half the inflow speed
    for _ in range(10):                            # gradient threshold: region >= 0.2 % of s0
        n, _ = dom.detect_region(g_thr, u_thr)
        if n >= 0.002 * N0:
            break
        g_thr *= 0.5
    h, every, margin = 0.5, 40, 4
    K, W = max(args.steps, every), args.warmup
    bid = dom.build_dynamic_scale(h, g_thr, u_thr, margin=margin)
    dom.step(W)
    dom.sync()
    # detection kernel alone: bytes = stored velocity (12 B) + flags (1 B) per node
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    dom.detect_region(g_thr, u_thr)
    e1.record(stream)
    e1.synchronize()
    t_det = e0.elapsed_time(e1) / 1e3
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(0)
    lu, alg, sizes = 0, 0, []
    torch.cuda.synchronize()
    clocks.start()
    ev0.record(stream)
    done = 0
    while done < K:
        bid = dom.build_dynamic_scale(h, g_thr, u_thr, margin=margin, replace_last=bid > 0)
        n = min(every, K - done)
        per_step = N0
        if bid > 0:
            i = dom.info(bid)
            nf = int(i.dims[0]) * int(i.dims[1]) * int(i.dims[2])
            per_step += int(i.substeps) * nf
            sizes.append(tuple(int(v) for v in i.dims))
        dom.step(n)
        lu += n * per_step
        done += n
    ev1.record(stream)
    ev1.synchronize()
    clk = clocks.stop()
    dom.sync()
    t = ev0.elapsed_time(ev1) / 1e3
    peak, peak_src = _peaks()
    achieved = lu * 249 / t / 1e9
    out = {"metric": "MLUPS", "value": lu / t / 1e6, "unit": "MLUPS", "steps": K,
           "ms_per_step": t / K * 1e3, "higher_is_better": True, "dtype": "f32",
           "config": {"workload": "dynamic256_fp32", "reference_nodes": int(N0), "h": h,
                      "rebuild_every": every, "g_threshold": g_thr, "u_threshold": u_thr,
                      "margin": margin, "dynamic_block_dims": sizes},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                        "kernel": "k_step over all blocks (249 B per update), rebuilds included"},
           "detect": {"ms_per_call": t_det * 1e3, "gb_per_s": N0 * 13 / t_det / 1e9,
                      "note": "k_detect_init + k_detect + read-back and synchronisation"},
           "clocks": clk}
    dom.close()
    if emit:
        print(json.dumps(out), flush=True)
    return out


def _line_spectra(u, mask_yz, x0, x1):
    """Mean power spectrum of the velocity fluctuation along x over the lines (y, z) in
    mask_yz, between x0 and x1 (line mean removed, Hann window, 3 components summed)."""
    import torch
    seg = u[:, :, :, x0:x1][:, mask_yz]                      # (3, lines, L)
    seg = seg - seg.mean(dim=-1, keepdim=True)
    win = torch.hann_window(x1 - x0, periodic=False, dtype=seg.dtype, device=seg.device)
    F = torch.fft.rfft(seg * win, dim=-1)
    return (F.real ** 2 + F.imag ** 2).sum(0).mean(0)        # E(k), k = 0 .. L/2


def run_ringing(args, emit=True):
    """Relaxation comparison on the flow past a sphere at the resolution and viscosity of
    Fig. 3 (196 x 98 x 98, nu = 1e-4, the sphere's surface as regularized walls): the same
    run with fixed high-order relaxation (phi = 1), adaptive relaxation from the lagged
    velocity gradient, and adaptive relaxation from the node's own strain rate.  Ringing is read from spectra: the power spectrum of the
    velocity fluctuation along the flow axis on lines outside the jet (distance > 30 from
    its axis, where the flow is smooth and high wavenumbers are artefacts) and inside it
    (distance < 12, the turbulence the relaxation should keep), every 250 steps; a run that
    blows up reports the step by which the library's divergence check caught it.  Every mode
    runs with two outer boundaries: Neumann (zero-gradient) faces on the box itself, and the
    paper's open-boundary setting (Sec. 4.2.4, 6.1), the box surrounded by a far-field block
    of spacing 2 reaching 32 reference units beyond it whose own faces are the Neumann ones.
    value = MLUPS of the adaptive (lagged-gradient) run with Neumann faces (the box alone)."""
    import torch

    import synth
    from paper_1807_02284_gb300 import lbm

    torch.cuda.set_device(0)
    sc = synth.ringing_channel()
    b = sc.blocks[0]
    nx, ny, nz = b.dims
    N = b.flags.size
    K = max(args.steps, 1)
    zz, yy = torch.meshgrid(torch.arange(nz), torch.arange(ny), indexing="ij")
    r = torch.sqrt((yy - 49.0) ** 2 + (zz - 49.0) ** 2)
    outer = ((r > 30.0) & (yy >= 4) & (yy < ny - 4) & (zz >= 4) & (zz < nz - 4)).cuda()
    jet = (r < 12.0).cuda()
    x0, x1 = 60, nx - 8                                       # downstream of the sphere
    res, clk, res_far = {}, None, {}
    fb = synth.far_block(b, 2.0, 32.0, seed=9, amp=0.0)
    runs = [(cfg, m) for cfg in ("neumann_faces", "far_field")
            for m in (("fixed", False, "lagged"), ("adaptive_lagged", True, "lagged"),
                      ("adaptive_local", True, "local"))]
    for cfg, (mode, adaptive, grad) in runs:
        stream = torch.cuda.Stream()
        dom = lbm.Domain(b.dims, sc.nu, periodic=sc.periodic, adaptive=adaptive,
                         c_src=sc.c_src, stream=stream, grad_mode=grad)
        dom.set_flags(b.flags)
        dom.set_walls((False,) * 6, obstacles=True)   # the sphere's surface: regularized walls
        dom.init_macro(b.u0.astype(np.float32), rho=b.rho0.astype(np.float32),
                       c=b.c0.astype(np.float32))
        far = cfg == "far_field"
        if far:                                       # at rest, no obstacles
            fid = dom.add_scale_block(fb.origin, fb.h, fb.dims)
            dom.init_macro(fb.u0.astype(np.float32), rho=fb.rho0.astype(np.float32),
                           c=fb.c0.astype(np.float32), block=fid)
        dom.step(args.warmup)
        dom.sync()
        sampler = ClockSampler(0) if (mode == "adaptive_lagged" and not far) else None
        if sampler:
            sampler.start()
        rec = {"steps": [], "outer_high_k_fraction": [], "jet_fluctuation_energy": [],
               "jet_high_k_fraction": []}
        t, done, diverged = 0.0, 0, None
        u = torch.empty(3 * N, dtype=torch.float32, device="cuda")
        while done < K:                 # chunks of 250 steps, spectra between the chunks
            n = min(250, K - done)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dom.step(n)
            e1.record(stream)
            e1.synchronize()
            t += e0.elapsed_time(e1) / 1e3
            done += n
            try:
                dom.read_field(lbm.LBM_FIELD_U, lbm.LBM_F32, out=u)
                dom.sync()
            except lbm.LBMError as ex:
                if ex.status != lbm.LBM_ERR_DIVERGED:
                    raise
                diverged = done
                break
            uu = u.view(3, nz, ny, nx).double()
            e_out = _line_spectra(uu, outer, x0, x1)
            e_jet = _line_spectra(uu, jet, x0, x1)
            kh = e_out.numel() // 2                           # half the Nyquist wavenumber
            rec["steps"].append(args.warmup + done)
            rec["outer_high_k_fraction"].append(float(e_out[kh:].sum() / e_out[1:].sum()))
            rec["jet_fluctuation_energy"].append(float(e_jet[1:].sum()))
            rec["jet_high_k_fraction"].append(float(e_jet[kh:].sum() / e_jet[1:].sum()))
        if sampler:
            clk = sampler.stop()
        dom.close()
        nodes = N + (fb.flags.size if far else 0)
        (res_far if far else res)[mode] = dict(
            mlups=nodes * done / t / 1e6,
            diverged_by_step=None if diverged is None else args.warmup + diverged, **rec)
    peak, peak_src = _peaks()
    alg, per_fluid = _algorithmic_bytes(b.flags, "fp32")
    ml = res["adaptive_lagged"]["mlups"]
    achieved = alg * ml * 1e6 / N / 1e9
    out = {"metric": "MLUPS", "value": ml, "unit": "MLUPS", "steps": K, "warmup": args.warmup,
           "higher_is_better": True, "dtype": "f32",
           "config": {"workload": "ringing196_fp32", "dims": list(b.dims), "nu": sc.nu,
                      "spectra": "velocity fluctuation along x, x in [60, 188), Hann window; "
                                 "outer: lines > 30 from the jet axis; jet: lines < 12; "
                                 "high k: above half the Nyquist wavenumber"},
           "ringing": dict(res, far_field=dict(res_far, block={"h": fb.h, "dims": list(fb.dims),
                                                                 "origin": list(fb.origin)})),
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                        "kernel": "k_step (adaptive, lagged gradient)"},
           "clocks": clk}
    if emit:
        print(json.dumps(out), flush=True)
    return out


def run_slab(args, emit=True):
    """The 256^3 plume cut into two z-slabs on one GPU (one stream for the slabs' steps, one
    for the packing): every step each slab steps the plane next to the cut first, packs its
    9 crossing populations, velocity, scalar and flags while its other planes step, and the
    neighbour unpacks them into its halo before the next step (halo planes themselves are not
    stepped).  The cost of the cut against the undivided plume; the exchange bytes are what
    one step would send between GPUs."""
    import torch

    import synth
    from paper_1807_02284_gb300 import sharding

    torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    sc = synth.plume(256)
    b = sc.blocks[0]
    world = 2
    stream = torch.cuda.Stream(device=dev)
    slabs = [sharding.SlabDomain(b.dims, sc.nu, rank=r, world=world, periodic=sc.periodic,
                                 adaptive=sc.adaptive, c_src=sc.c_src, stream=stream)
             for r in range(world)]
    for s in slabs:
        s.set_flags(b.flags)
        s.init_macro(b.u0, rho=b.rho0, c=b.c0)
    K, W = args.steps, args.warmup
    sharding.step_local(slabs, W)
    for s in slabs:
        s.sync()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dev)
    torch.cuda.synchronize()
    clocks.start()
    ev0.record(stream)
    sharding.step_local(slabs, K)
    ev1.record(stream)
    ev1.synchronize()
    clk = clocks.stop()
    for s in slabs:
        s.sync()
    t = ev0.elapsed_time(ev1) / 1e3
    N = b.flags.size
    sends = [(s.plan.rank, z, peer, tag) for s in slabs for (k, z, peer, tag) in s.plan.transfers()
             if k == "send"]
    xbytes = sum(slabs[r].dom.plane_bytes(sharding.DIRECTION[tag]) for r, _, _, tag in sends)
    alg, per_fluid = _algorithmic_bytes(b.flags, "fp32")
    peak, peak_src = _peaks()
    achieved = alg / (t / K) / 1e9
    halo_nodes = 0                   # halo planes are unpacked, not stepped
    out = {"metric": "MLUPS", "value": N * K / t / 1e6, "unit": "MLUPS", "n_gpus": 1,
           "steps": K, "warmup": W, "ms_per_step": t / K * 1e3, "higher_is_better": True,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": "plume256_slab2", "slabs": world,
                      "slab_planes": [s.plan.z1 - s.plan.z0 for s in slabs],
                      "lattice_updates_per_step": int(N),
                      "halo_node_updates_per_step": int(halo_nodes),
                      "exchange_bytes_per_step": int(xbytes),
                      "l2": "inputs larger than L2"},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                        "kernel": "k_step on both slabs (send plane, then the other planes) + "
                                  "k_plane pack (overlapped) / unpack (undivided-domain "
                                  "algorithmic bytes over the whole step)"},
           "gpu_launches": K * (world + 3 * len(sends)),
           "clocks": clk}
    for s in slabs:
        s.close()
    if emit:
        print(json.dumps(out), flush=True)
    return out


def _variants(args):
    """Measured summaries of the other hot-path variants for the default bench line."""
    import copy
    import io
    from contextlib import redirect_stdout

    res = {}
    for name, fn, steps, warm in (("plume256_fp16", run_ours, 100, 10),
                                  ("plume256_local", run_ours, 100, 10),
                                  ("plume256_walls", run_ours, 100, 10),
                                  ("multiscale3", run_ours, 48, 48),
                                  ("multiscale3_regwall", run_ours, 48, 48),
                                  ("dynamic256", run_dynamic, 200, 10),
                                  ("farfield256", run_ours, 96, 96),
                                  ("batch64", run_batch, 100, 10),
                                  ("adjoint128", run_adjoint, 200, 0),
                                  ("ringing196", run_ringing, 3000, 10),
                                  ("plume256_regwall", run_ours, 100, 10),
                                  ("plume256_slab2", run_slab, 100, 10)):
        a = copy.copy(args)
        a.workload, a.steps, a.warmup, a.no_cpu_baseline = name, steps, warm, True
        buf = io.StringIO()
        try:
            with redirect_stdout(buf):
                fn(a)
            d = json.loads(buf.getvalue().strip().splitlines()[-1])
            res[name] = {k: d[k] for k in ("value", "unit", "ms_per_step", "roofline", "e2e",
                                           "forward_with_tape_mlups", "config", "detect",
                                           "ringing")
                         if k in d}
        except Exception as ex:  # report, do not hide
            res[name] = {"error": f"{type(ex).__name__}: {ex}"}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--workload", default="plume256",
                    choices=["plume256", "plume256_fp16", "plume128", "plume128_fp16",
                             "plume192", "plume192_fp16",
                             "multiscale3", "batch64", "adjoint128", "adjoint64",
                             "plume256_local", "dynamic256", "farfield256", "plume256_walls",
                             "ringing196", "plume256_regwall", "plume256_slab2",
                             "multiscale3_regwall"])
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the FP16 / multi-scale / batch / adjoint summaries")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=24.0)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in ("adjoint128", "adjoint64"):
        run_adjoint(args)
    elif args.workload == "batch64":
        run_batch(args)
    elif args.workload == "dynamic256":
        run_dynamic(args)
    elif args.workload == "ringing196":
        run_ringing(args)
    elif args.workload == "plume256_slab2":
        run_slab(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
