#!/usr/bin/env python
"""Benchmark of the HDG trace-solver hot path (one GB300 per rank).

Workload (default): HDG linear elasticity (E = 1, nu = 0.3) on a 32^3 hex mesh
whose interior vertices are moved by up to 0.2h (seed 3), Q2 tensor basis
(27 trace dofs per face, 162 x 162 condensed element blocks), 2,571,264 trace
unknowns, 8 right-hand sides from seeded N(0,1) nodal body forces; GMRES(50)
with block-Jacobi + degree-4 Chebyshev preconditioning to a true FP64
relative residual of 1e-8 for every right-hand side.

One step = one pass of the whole hot path: the element blocks generated on
the device from the vertices and condensed (hdg_condense_hex), face-based
assembly, preconditioner set-up (block-Jacobi inverses, the Arnoldi cycle of
the Chebyshev bounds), GMRES to 1e-8, element recovery.  `value` is the step
with the mixed-precision solve (FP32 or BF16 blocks, FP64 Krylov basis and
residuals); the same step with the plain FP64 solve, the additive-Schwarz
variants, the 16^3 Q3 Poisson step and the serving stream are measured beside
it.

Prints ONE JSON line (rank 0).  Several ranks run independent replicas (the
path is not sharded); timings are the max over ranks.
`--impl reference` times the FP64 CPU oracle (test infrastructure) on a
bounded sample of the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = 'time to 1e-8 rel. residual (mixed vs FP64); block-matvec GB/s; p99 latency'
WORKLOAD = 'HDG Poisson, unit cube, 16^3 hex, Q3 (16 dofs/face, 96x96 element blocks), sin-product MMS, 1 RHS'
WORKLOAD3 = ('HDG linear elasticity (E=1, nu=0.3), 32^3 hex with interior vertices perturbed by up to 0.2h '
             '(seed 3), Q2 (27 dofs/face, 162x162 element blocks), 8 RHS from N(0,1) nodal body forces '
             '(seeds 300-307), BJ + Chebyshev(4) GMRES(50) to 1e-8')
ORACLE_SAMPLE_N = 6      # the oracle's bounded sample of the elasticity workload: 6^3 elements


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=5)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--n', type=int, default=16)
    ap.add_argument('--k', type=int, default=3)
    ap.add_argument('--no-e2e', action='store_true')
    ap.add_argument('--no-cpu', action='store_true')
    ap.add_argument('--no-graphs', action='store_true', help='launch GMRES iterations one by one')
    ap.add_argument('--serving-requests', type=int, default=256,
                    help='requests of the serving stream per load point, timed beside the step (0: none)')
    ap.add_argument('--lanes', type=int, default=4, help='concurrent requests of the serving loop')
    ap.add_argument('--serving-mixed', choices=['refinement', 'restarted'], default='restarted',
                    help='mixed-precision mode of the serving solves')
    ap.add_argument('--serving-cold', dest='serving_warm', action='store_false',
                    help='start the serving stream without slots (default: one slot per shape)')
    ap.add_argument('--serving-budget-gb', type=float, default=160.0)
    ap.add_argument('--mesh-n', type=int, default=0, help='mesh size of --workload (0: 40 / 32)')
    ap.add_argument('--max-iters', type=int, default=3000, help='GMRES iteration cap of --workload solves')
    ap.add_argument('--mixed-mode', choices=['restarted', 'refinement', 'precond'], default='restarted',
                    help='mixed-precision mode of the value leg: restarted (FP32 cycles, FP64 residual at each '
                         'restart), refinement (FP64 refinement around FP32 inner solves) or precond (FP64 '
                         'operator and Krylov, preconditioner in FP32)')
    ap.add_argument('--poly-prec', choices=['fp32', 'bf16'], default='fp32',
                    help='storage of K inside the Chebyshev polynomial of the mixed legs')
    ap.add_argument('--no-asm', action='store_true', help='skip the additive-Schwarz legs of the default step')
    ap.add_argument('--no-config2', action='store_true', help='skip the 16^3 Q3 Poisson leg of the default step')
    ap.add_argument('--workload', choices=['step3', 'poisson16', 'elasticity32', 'cdr40', 'beam', 'beamcheck', 'tets',
                                           'burgers'],
                    default='step3',
                    help='step3: the step above (default); poisson16: the same step on the 16^3 Q3 Poisson '
                         'workload with resident element blocks; elasticity32 / cdr40: solver and kernel measurements '
                         'on the 32^3 perturbed Q2 elasticity (8 RHS) and 40^3 Q2 5-component CDR (4 RHS) '
                         'problems; beam: the cantilever beam runs of Sec. 6.2 (BJ, BJ-PP(10), ASM, '
                         'ASM-PP(10), GMRES(50) to 1e-6) over k at N_E = 320 and over N_E at k = 3; '
                         'tets: the tetrahedral Poisson runs of Sec. 6.1 (BJ-PP(10/20), ASM-PP(10/20)) on a '
                         'synthetic obstacle mesh of 6 n^3 Kuhn tetrahedra (--mesh-n, default 26: 104,160); '
                         'one JSON line')
    ap.add_argument('--tet-ks', default='1,2,3,4', help='polynomial degrees of --workload tets')
    ap.add_argument('--burgers-cases', default='1:16,1:32,1:64,1:128,2:16,2:32,2:64,2:128,3:16,3:32,3:64,3:128,'
                                               '4:16,4:32,4:64,4:128',
                    help='k:1/h pairs of --workload burgers (Sec. 6.1 Table 1: steady viscous Burgers, damped '
                         'Newton with BJ, BJ-PP(10), ASM, ASM-PP(10) GMRES(50) to 1e-6)')
    ap.add_argument('--beam-cases', default='4:1,4:2,4:3,4:4,2:3,6:3,8:3',
                    help='n:k pairs of --workload beam (5n x n x n hexahedra, Q^k)')
    ap.add_argument('--k32-config', default='',
                    help='with --profile matvec3: run the FP32 product of K in this launch configuration '
                         '(kind,slot parts,CTAs per SM, e.g. 8,1,32) instead of the tuned one')
    ap.add_argument('--profile', choices=['condense', 'matvec', 'solve-mixed', 'solve-fp64', 'generate', 'step3',
                                          'matvec3'],
                    default=None,
                    help='set up the workload and run only one hdg_condense call (condense), one FP64 and '
                         'one FP32 hdg_apply_K call (matvec), one solve (solve-*) or two hdg_hex_blocks calls '
                         '(generate: the element blocks generated on the device), or two mixed steps of the '
                         'default workload (step3, --mesh-n sets its size), or one FP64, FP32 and BF16 '
                         'hdg_apply_K call on the default workload after autotuning (matvec3), for profilers; '
                         'no JSON')
    return ap.parse_args()


# Sources of the FP32 block-row kernel (R = 8) whose DRAM traffic a committed
# ncu summary records; the summary's figure is reported only while these files
# hash to the value recorded beside it.
TRAFFIC_SOURCES = ['paper_2512_13619_gb300/csrc/k_blockrow.cuh', 'paper_2512_13619_gb300/csrc/k_blockrow_f32_wide.cu',
                   'paper_2512_13619_gb300/csrc/k_poly.cuh', 'paper_2512_13619_gb300/csrc/hdg_common.cuh']
TRAFFIC_SUMMARY = 'profiles/blockrow_vec_fp32_elasticity_32_q2_r8_traffic.md'


def sources_sha256(paths):
    import hashlib
    h = hashlib.sha256()
    root = os.path.dirname(os.path.abspath(__file__))
    for rel in paths:
        with open(os.path.join(root, rel), 'rb') as f:
            h.update(f.read())
    return h.hexdigest()


def profiled_traffic(cfg):
    """DRAM bytes (read + write) per launch of the FP32 block-row kernel on
    the 32^3 elasticity workload from the committed ncu summary, or None when
    the summary is absent, was taken with another configuration, or the
    kernel's sources changed since."""
    root = os.path.dirname(os.path.abspath(__file__))
    try:
        text = open(os.path.join(root, TRAFFIC_SUMMARY)).read()
    except OSError:
        return None, 'no ncu summary'
    rec = {}
    for line in text.splitlines():
        if line.startswith('traffic_record:'):
            for tok in line.split()[1:]:
                k, _, v = tok.partition('=')
                rec[k] = v
    if not rec:
        return None, 'no record in the ncu summary'
    if rec.get('cfg') != ','.join(str(c) for c in cfg):
        return None, 'tuned configuration %s differs from the profiled %s' % (list(cfg), rec.get('cfg'))
    if rec.get('sources_sha256') != sources_sha256(TRAFFIC_SOURCES):
        return None, 'kernel sources changed since the ncu capture'
    return int(rec['dram_bytes_per_launch']), TRAFFIC_SUMMARY


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, 'MEASURED_PEAKS.json')))
    except Exception:
        return {'hbm_gbs': 6800.0, 'bf16_tflops': 1900.0, '_fallback': True}


# DRAM read + write of the tensor-core condensation products of one 16^3 Q3
# condensation: ncu capture of the 8 launches of the same kernel on the 8^3
# Q3 case (512 elements, 900.2 MB read + 96.6 MB written), scaled by the
# element count (x 8).  Taken with the kernel as committed; to be set to None
# when the kernel changes.
OZAKI_DRAM_BYTES_PER_CONDENSATION = int((900.2e6 + 96.6e6) * 8)

# FP64 ALU peak: 152 SMs x 2.07 GHz x 4 FP64 FLOP/clk/SM (nominal 1.25 TFLOP/s)
FP64_ALU_PEAK_TFLOPS = 152 * 2.07e9 * 4 / 1e12


class Clocks:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""
    FIELDS = 'index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,' \
             'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,' \
             'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap'

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(['nvidia-smi', '-i', str(self.gpu), '--query-gpu=' + self.FIELDS,
                                          '--format=csv,noheader,nounits', '-lms', '200'],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        for ln in self.lines:
            f = [x.strip() for x in ln.split(',')]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == 'active':
                    reasons.add(nm)
        if not sm:
            return None
        sm.sort()
        return {'sm_mhz': sm[len(sm) // 2], 'sm_max_mhz': max(mx), 'samples': len(sm), 'reasons': sorted(reasons)}


def dist_setup():
    ws = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    return ws, rank, local


def max_over_ranks(value, dist=None, device=None):
    """The largest `value` over the ranks of the process group (the value
    itself without one): every rank times its own replica, the job's time is
    the slowest rank's.  NCCL reduces a device tensor, gloo a host tensor."""
    if dist is None:
        return float(value)
    import torch
    dev = device if dist.get_backend() == 'nccl' else 'cpu'
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def condense_flops(w):
    """Algorithmic FP64 flops of the batched condensation per element
    (Eqs. w16-w22 as implemented: inverses by Gauss-Jordan, 2n^3)."""
    PE, D, M, PF, nl, R = w.PE, w.D, w.M, w.PF, w.n_lfe, w.R
    MPE, nlPF, nlb = M * PE, nl * PF, nl * M * PF
    f = 2 * PE ** 3 + D * 2 * PE ** 3 + D * 2 * PE ** 2 * nlPF
    f += 2 * MPE * MPE * D * PE + 2 * MPE * nlb * D * PE + 2 * nlb * MPE * D * PE + 2 * nlb * nlb * D * PE
    f += 2 * MPE ** 3 + 2 * MPE ** 2 * (nlb + R) + 2 * nlb * MPE * (nlb + R)
    return f


def tensor_digit_flops(w):
    """Tensor-core flops of the condensation products per element: the
    products with N >= 16 (all but the right-hand-side columns) run as 36
    BF16 digit products of 2 M N K flops each."""
    PE, D, M, PF, nl = w.PE, w.D, w.M, w.PF, w.n_lfe
    MPE, nlPF, nlb = M * PE, nl * PF, nl * M * PF
    shapes = [(PE, PE, PE, D), (PE, nlPF, PE, D), (MPE, PE, D * PE, M), (MPE, nlPF, D * PE, M),
              (nlb, PE, D * PE, M), (nlb, nlPF, D * PE, M), (MPE, nlb, MPE, 1), (nlb, nlb, MPE, 1)]
    return sum(36 * 2 * m * n * k * c for m, n, k, c in shapes if n >= 16 and k <= 192)


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dev = torch.device('cuda', local)
    import __graft_entry__
    __graft_entry__.build()
    from hdg_inputs import workloads as W
    from paper_2512_13619_gb300 import driver, _lib as L

    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl', device_id=dev)

    w = W.hex_poisson(n=args.n, k=args.k)
    blk = w.blocks()
    names = driver.BLOCK_NAMES
    host = {k: torch.from_numpy(np.ascontiguousarray(blk[k])).pin_memory() for k in names}
    dblk = {k: host[k].to(dev) for k in names}
    uD_host = torch.from_numpy(w.uhat_dirichlet()).pin_memory()
    uD_dev = uD_host.to(dev)
    in_bytes = sum(v.numel() * 8 for v in host.values()) + uD_host.numel() * 8
    R = w.R
    o_mixed = driver.opts(restart=50, rtol=1e-8, pc='bj', inner='fp32', inner_rtol=1e-4, max_iters=5000)
    o_fp64 = driver.opts(restart=50, rtol=1e-8, pc='bj', inner='fp64', max_iters=5000)
    o_mixed_rs = driver.opts(restart=50, rtol=1e-8, pc='bj', inner='fp32', max_iters=5000, max_outer=-1)
    p = driver.Problem.from_workload(w, local)
    if args.no_graphs:
        L.hdg_set_graphs(p.h, 0)
    u_dev = torch.empty((w.n_elem, w.M * w.PE, R), dtype=torch.float64, device=dev)
    q_dev = torch.empty((w.n_elem, w.M * w.D * w.PE, R), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    st = stream.cuda_stream
    infos = {}

    def step(o, tag, phases=None):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)] if phases is not None else None
        if ev: ev[0].record()
        driver.check(L.hdg_condense(p.h, 0, w.n_elem, *[dblk[k] for k in names], 1, st), 'condense')
        driver.check(L.hdg_set_dirichlet(p.h, uD_dev, 1, st), 'dirichlet')
        driver.check(L.hdg_assemble(p.h, o, st), 'assemble')
        driver.check(L.hdg_setup_precond(p.h, o, None, st), 'setup')
        if ev: ev[1].record()
        info = L.hdg_solve_info()
        s = L.hdg_solve(p.h, o, st, info)
        if s != 0:
            raise RuntimeError('%s solve: %s rel=%g' % (tag, L.hdg_status_str(s), info.rel_resid))
        if ev: ev[2].record()
        driver.check(L.hdg_recover(p.h, u_dev, q_dev, 1, st), 'recover')
        if ev:
            ev[3].record()
            phases.append(ev)
        infos[tag] = (info.iters, info.outer, info.rel_resid)

    def timed(o, tag, K, timing=False):
        for _ in range(args.warmup):
            step(o, tag)
        torch.cuda.synchronize(dev)
        if dist: dist.barrier()
        torch.cuda.synchronize(dev)
        L.hdg_set_timing(p.h, 1 if timing else 0)
        phases = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0 = L.hdg_launch_count()
        e0.record()
        for _ in range(K):
            step(o, tag, phases)
        e1.record()
        torch.cuda.synchronize(dev)
        n1 = L.hdg_launch_count()
        ms = e0.elapsed_time(e1) / K
        ph = {'setup': 0.0, 'solve': 0.0, 'recover': 0.0}
        for ev in phases:
            ph['setup'] += ev[0].elapsed_time(ev[1]) / K
            ph['solve'] += ev[1].elapsed_time(ev[2]) / K
            ph['recover'] += ev[2].elapsed_time(ev[3]) / K
        tm = [L.hdg_get_timing(p.h, kind) for kind in range(3)]
        L.hdg_set_timing(p.h, 0)
        ms = max_over_ranks(ms, dist, dev)
        return ms, ph, (n1 - n0) / K, tm

    o_fp64_10 = driver.opts(restart=50, rtol=1e-10, pc='bj', inner='fp64', max_iters=5000)
    clk = Clocks(local)
    clk.start()
    ms_fp64, ph_fp64, launches, _ = timed(o_fp64, 'fp64', args.steps)
    ms_mixed, ph_mixed, launches_mixed, _ = timed(o_mixed, 'mixed', args.steps)
    ms_fp64_10, _, _, _ = timed(o_fp64_10, 'fp64_1e-10', args.steps)
    ms_mixed_rs, ph_mixed_rs, _, _ = timed(o_mixed_rs, 'mixed_restarted', args.steps)

    # block matvec alone: the library's CUDA events around each block-row
    # launch on the launching stream (hdg_set_timing), an L2 flush (a 256 MiB
    # write) between launches, after 3 warm-up launches
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    xv = torch.randn(p.n_dof * R, dtype=torch.float64, device=dev)
    yv = torch.empty_like(xv)
    mv_ms = {}
    for prec in (L.HDG_FP64, L.HDG_FP32):
        for _ in range(3):
            driver.check(L.hdg_apply_K(p.h, prec, xv, yv, st), 'apply_K')
        torch.cuda.synchronize(dev)
        nrep = max(10, args.steps * 4)
        L.hdg_set_timing(p.h, 1)
        for _ in range(nrep):
            flush.fill_(1.0)
            driver.check(L.hdg_apply_K(p.h, prec, xv, yv, st), 'apply_K')
        torch.cuda.synchronize(dev)
        _, tms, nl = L.hdg_get_timing(p.h, prec)
        L.hdg_set_timing(p.h, 0)
        mv_ms[prec] = (tms / max(nl, 1), nl)
    clocks = clk.stop()

    # condensation alone (the dominant kernels: the tensor-core products,
    # the FP64 inverses)
    torch.cuda.synchronize(dev)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record()
    for _ in range(args.steps):
        driver.check(L.hdg_condense(p.h, 0, w.n_elem, *[dblk[k] for k in names], 1, st), 'condense')
    c1.record()
    torch.cuda.synchronize(dev)
    ms_cond = c0.elapsed_time(c1) / args.steps
    cflops = condense_flops(w) * w.n_elem
    # the tensor-core products alone: library events around each of their launches
    L.hdg_set_timing(p.h, 1)
    for _ in range(args.steps):
        driver.check(L.hdg_condense(p.h, 0, w.n_elem, *[dblk[k] for k in names], 1, st), 'condense')
    _, tc_ms, tc_n = L.hdg_get_timing(p.h, 3)
    L.hdg_set_timing(p.h, 0)
    tc_ms_step = tc_ms / args.steps
    tc_flops = tensor_digit_flops(w) * w.n_elem
    # the same condensation with the element blocks generated on the device
    # from the vertices (hdg_condense_hex); beside the step, not part of it
    gverts, gperm, nquad = driver.hex_geometry_inputs(w)
    gverts, gperm = torch.from_numpy(gverts).to(dev), torch.from_numpy(gperm).to(dev)
    gphys, _keep = L.physics(w.phys.Cq, w.phys.Cu, w.phys.Rr, w.phys.tau)

    def gen_condense():
        driver.check(L.hdg_condense_hex(p.h, 0, w.n_elem, nquad, gverts, gperm, gphys, dblk['ru'], dblk['ruh'], 1,
                                        st), 'condense_hex')
    gen_condense()
    torch.cuda.synchronize(dev)
    c0.record()
    for _ in range(args.steps):
        gen_condense()
    c1.record()
    torch.cuda.synchronize(dev)
    ms_gen_cond = c0.elapsed_time(c1) / args.steps

    # end to end through the C ABI from pinned host buffers (inputs in, trace + u + q out)
    e2e = None
    if not args.no_e2e:
        uh_host = torch.empty((w.n_face, w.M * w.PF, R), dtype=torch.float64).pin_memory()
        u_host = torch.empty((w.n_elem, w.M * w.PE, R), dtype=torch.float64).pin_memory()
        q_host = torch.empty((w.n_elem, w.M * w.D * w.PE, R), dtype=torch.float64).pin_memory()

        def e2e_step():
            driver.check(L.hdg_condense(p.h, 0, w.n_elem, *[host[k] for k in names], 0, st), 'condense')
            driver.check(L.hdg_set_dirichlet(p.h, uD_host, 0, st), 'dirichlet')
            driver.check(L.hdg_assemble(p.h, o_fp64, st), 'assemble')
            driver.check(L.hdg_setup_precond(p.h, o_fp64, None, st), 'setup')
            info = L.hdg_solve_info()
            s = L.hdg_solve(p.h, o_fp64, st, info)
            if s != 0:
                raise RuntimeError('e2e solve: ' + L.hdg_status_str(s))
            driver.check(L.hdg_get_trace(p.h, uh_host, 0, st), 'trace')
            driver.check(L.hdg_recover(p.h, u_host, q_host, 0, st), 'recover')
        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize(dev)
        if dist: dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize(dev)
        e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        e_ms = max_over_ranks(e_ms, dist, dev)
        out_bytes = (uh_host.numel() + u_host.numel() + q_host.numel()) * 8
        e2e = {'value': round(e_ms, 3), 'unit': 'ms', 'h2d_bytes_per_step': int(in_bytes),
               'd2h_bytes_per_step': int(out_bytes)}

    pk = peaks()
    fd = w.face_dirichlet
    nfree_e = (fd[w.mesh.elem_face] == 0).sum(axis=1)
    nnzb = int((nfree_e ** 2).sum() - w.n_free)      # nonzero b x b blocks of K
    b = w.M * w.PF
    mv = {}
    for prec, name, sz in ((0, 'fp64', 8), (1, 'fp32', 4)):
        avg, n = mv_ms[prec]
        # FP64 blocks: K + x + y (FP64).  FP32 blocks: K + the FP32 copy of x
        # (read) + y (FP64); the events bracket the block-row kernel alone
        by = nnzb * b * b * sz + p.n_dof * R * (16 if prec == 0 else 12)
        gbs = by / avg / 1e6
        tf = 2 * nnzb * b * b * R / avg / 1e9
        mv[name] = {'avg_ms': round(avg, 5), 'launches': int(n), 'bytes_per_launch': int(by),
                    'gbs': round(gbs, 1), 'frac_hbm': round(gbs / pk['hbm_gbs'], 3), 'tflops': round(tf, 3),
                    'frac_fp64_alu': round(tf / FP64_ALU_PEAK_TFLOPS, 3) if prec == 0 else None,
                    'timing': 'CUDA events around each block-row launch, L2 flushed between launches'}
    achieved = tc_flops / tc_ms_step / 1e9
    roof = {'kernel': 'gemm_ozaki_kernel (+ its exponent pass): FP64-accurate condensation products on the '
                      'BF16 tensor cores, 36 digit products per FP64 product',
            'bound': 'tensor', 'achieved': round(achieved, 2), 'peak': pk['bf16_tflops'],
            'unit': 'TFLOP/s', 'frac': round(achieved / pk['bf16_tflops'], 4),
            'traffic': OZAKI_DRAM_BYTES_PER_CONDENSATION if (args.n, args.k) == (16, 3) else None,
            'traffic_unit': 'DRAM bytes per condensation (all 32 launches)',
            'flops_per_step': int(tc_flops), 'ms_per_step': round(tc_ms_step, 3),
            'launches_per_step': tc_n // args.steps,
            'peak_source': 'MEASURED_PEAKS.json bf16_tflops (burst; the products are timed in their own loop)'
                           if not pk.get('_fallback') else 'fallback 1.9 PFLOP/s bf16',
            'condensation': {'ms_per_step': round(ms_cond, 3), 'fp64_flops_per_step': int(cflops),
                             'fp64_equivalent_tflops': round(cflops / ms_cond / 1e9, 3),
                             'vs_fp64_alu_peak': round(cflops / ms_cond / 1e9 / FP64_ALU_PEAK_TFLOPS, 3)}}
    out = {
        'metric': METRIC, 'value': round(ms_fp64, 3), 'unit': 'ms', 'n_gpus': ws, 'steps': args.steps,
        'warmup': args.warmup, 'ms_per_step': round(ms_fp64, 3), 'higher_is_better': False, 'scaling': 'weak',
        'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic',
        'config': {'workload': WORKLOAD, 'n_elem': w.n_elem, 'n_dof': p.n_dof, 'precond': 'block-Jacobi',
                   'restart': 50, 'rtol': 1e-8, 'rhs': R, 'solve': 'FP64 GMRES (plain path)',
                   'l2': 'inputs larger than L2 (%.2f GB element blocks read per step)' % (in_bytes / 1e9),
                   'parallelism': 'replicas' if ws > 1 else 'single GPU'},
        'mixed_ms_per_step': round(ms_mixed, 3),
        'speedup_mixed_vs_fp64': round(ms_fp64 / ms_mixed, 3),
        'mixed_restarted_ms_per_step': round(ms_mixed_rs, 3),
        'speedup_mixed_restarted_vs_fp64': round(ms_fp64 / ms_mixed_rs, 3),
        'fp64_to_1e-10_ms_per_step': round(ms_fp64_10, 3),
        'generated_condense_ms': round(ms_gen_cond, 3),
        'generated_condense_note': 'condensation with the element blocks generated on the device from the '
                                   'vertices (hdg_condense_hex), timed beside the step; the step reads resident '
                                   'blocks',
        'phases_ms': {'mixed': {k: round(v, 3) for k, v in ph_mixed.items()},
                      'mixed_restarted': {k: round(v, 3) for k, v in ph_mixed_rs.items()},
                      'fp64': {k: round(v, 3) for k, v in ph_fp64.items()}, 'condense': round(ms_cond, 3)},
        'iterations': {k: {'gmres': v[0], 'refinement': v[1], 'rel_resid': v[2]} for k, v in infos.items()},
        'aggregate_solves_per_s': round(ws * 1000.0 / ms_fp64, 3),
        'block_matvec': mv,
        'roofline': roof,
        'gpu_launches': int(round(launches)),
        'clocks': clocks,
    }
    if e2e:
        out['e2e'] = e2e
    p.close()
    if args.serving_requests > 0:
        out['serving'] = serving_leg(args, local)
    if rank == 0 and not args.no_cpu:
        out['cpu_baseline'] = cpu_baseline(args, w, blk)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return out


def nonzero_blocks(w):
    """Real nonzero b x b blocks of K: sum over elements of (free faces)^2
    minus the free faces (each diagonal block is shared by two elements)."""
    fd = w.face_dirichlet
    nfree_e = (fd[w.mesh.elem_face] == 0).sum(axis=1)
    return int((nfree_e ** 2).sum() - w.n_free)


def run_step3(args, ws, rank, local):
    """The default step on the 32^3 perturbed Q2 elasticity workload (8 RHS):
    device-generated blocks, condensation, assembly, BJ + Chebyshev(4) set-up,
    GMRES(50) to 1e-8 (mixed and FP64), recovery."""
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dev = torch.device('cuda', local)
    import __graft_entry__
    __graft_entry__.build()
    from hdg_inputs import workloads as W
    from paper_2512_13619_gb300 import driver, _lib as L

    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl', device_id=dev)

    t_in = time.perf_counter()
    n = args.mesh_n or 32
    w = W.hex_elasticity(n=n, k=2, R=8)
    verts, perm, nquad = driver.hex_geometry_inputs(w)
    ru, ruh = w.load_vectors()
    uD = np.zeros((w.n_face, w.M * w.PF, w.R))
    host = {k: torch.from_numpy(v).pin_memory() for k, v in
            (('verts', verts), ('perm', perm), ('ru', ru), ('ruh', ruh), ('uD', uD))}
    dvc = {k: v.to(dev) for k, v in host.items()}
    phys, _keep = L.physics(w.phys.Cq, w.phys.Cu, w.phys.Rr, w.phys.tau)
    v0 = torch.from_numpy(w.random_vector(31)).to(dev)      # start vector of the Chebyshev bounds' Arnoldi cycle
    t_in = time.perf_counter() - t_in
    R = w.R
    p = driver.Problem.from_workload(w, local)
    if args.no_graphs:
        L.hdg_set_graphs(p.h, 0)
    u_dev = torch.empty((w.n_elem, w.M * w.PE, R), dtype=torch.float64, device=dev)
    q_dev = torch.empty((w.n_elem, w.M * w.D * w.PE, R), dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev).cuda_stream
    in_bytes = sum(v.numel() * v.element_size() for v in host.values())
    mo = {'restarted': -1, 'refinement': 20, 'precond': -2}

    def o_of(pc, poly, deg, inner, mode='restarted', pprec='fp32'):
        return driver.opts(restart=50, rtol=1e-8, pc=pc, poly=poly, degree=deg, inner=inner,
                           poly_prec=pprec if inner != 'fp64' else 'fp64', inner_rtol=1e-4, max_iters=3000,
                           max_outer=mo[mode] if inner != 'fp64' else 20)
    legs = {
        'mixed': ('BJ + Chebyshev(4), %s mixed, FP32 blocks, %s polynomial' % (args.mixed_mode, args.poly_prec.upper()),
                  o_of('bj', 'chebyshev', 4, 'fp32', args.mixed_mode, args.poly_prec)),
        'fp64': ('BJ + Chebyshev(4), plain FP64', o_of('bj', 'chebyshev', 4, 'fp64')),
    }
    if not args.no_asm:
        legs['asm_mixed'] = ('ASM (one-element patches), restarted mixed, FP32 blocks',
                             o_of('asm', None, 0, 'fp32', 'restarted'))
        legs['asm_fp64'] = ('ASM (one-element patches), plain FP64', o_of('asm', None, 0, 'fp64'))
    infos = {}

    def step(o, tag, src, on_device, phases=None, outs=None):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if phases is not None else None
        if ev: ev[0].record()
        driver.check(L.hdg_condense_hex(p.h, 0, w.n_elem, nquad, src['verts'], src['perm'], phys, src['ru'],
                                        src['ruh'], on_device, st), 'condense_hex')
        driver.check(L.hdg_set_dirichlet(p.h, src['uD'], on_device, st), 'dirichlet')
        driver.check(L.hdg_assemble(p.h, o, st), 'assemble')
        driver.check(L.hdg_setup_precond(p.h, o, v0, st), 'setup')
        if ev: ev[1].record()
        info = L.hdg_solve_info()
        s_ = L.hdg_solve(p.h, o, st, info)
        if s_ != 0:
            raise RuntimeError('%s solve: %s rel=%g' % (tag, L.hdg_status_str(s_), info.rel_resid))
        if ev: ev[2].record()
        if outs is None:
            driver.check(L.hdg_recover(p.h, u_dev, q_dev, 1, st), 'recover')
        else:
            driver.check(L.hdg_get_trace(p.h, outs[0], 0, st), 'trace')
            driver.check(L.hdg_recover(p.h, outs[1], outs[2], 0, st), 'recover')
        if ev:
            ev[3].record()
            phases.append(ev)
        infos[tag] = (info.iters, info.outer, info.rel_resid)

    def timed(o, tag, K, W_):
        for _ in range(W_):
            step(o, tag, dvc, 1)
        torch.cuda.synchronize(dev)
        if dist: dist.barrier()
        torch.cuda.synchronize(dev)
        phases = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0 = L.hdg_launch_count()
        e0.record()
        for _ in range(K):
            step(o, tag, dvc, 1, phases)
        e1.record()
        torch.cuda.synchronize(dev)
        n1 = L.hdg_launch_count()
        ms = e0.elapsed_time(e1) / K
        ph = {'setup': 0.0, 'solve': 0.0, 'recover': 0.0}
        for ev in phases:
            ph['setup'] += ev[0].elapsed_time(ev[1]) / K
            ph['solve'] += ev[1].elapsed_time(ev[2]) / K
            ph['recover'] += ev[2].elapsed_time(ev[3]) / K
        ms = max_over_ranks(ms, dist, dev)
        print('step3 %s: %.1f ms per step (%s), iterations %s' % (tag, ms, {k: round(v, 1) for k, v in ph.items()},
                                                                    infos[tag]), file=sys.stderr, flush=True)
        return ms, ph, (n1 - n0) / K

    # set-up: one untimed step of each preconditioner, then the autotuner
    # picks the block-row launch configurations (K at every stored precision,
    # BJ and ASM; cached per block shape)
    tuning = {}
    for tag in [t for t in ('asm_mixed', 'mixed') if t in legs]:
        o = legs[tag][1]
        step(o, tag, dvc, 1)
        if tag == 'mixed':
            driver.check(L.hdg_assemble(p.h, o_of('bj', None, 0, 'fp32', 'restarted', 'bf16'), st), 'assemble')
            driver.check(L.hdg_setup_precond(p.h, o, v0, st), 'setup')
        driver.check(L.hdg_autotune(p.h, 10, 0, st), 'autotune')
    for op, opn in ((0, 'K'), (1, 'bj'), (2, 'asm')):
        for prec, pn in ((0, 'fp64'), (1, 'fp32'), (2, 'bf16')):
            _, cfg, us, us0 = L.hdg_get_tuning(p.h, op, prec)
            if us > 0:
                tuning['%s_%s' % (opn, pn)] = {'cfg': list(cfg), 'us_tuned': round(us, 1), 'us_default': round(us0, 1)}

    clk = Clocks(local)
    clk.start()
    res = {}
    ms_val, ph_val, launches = timed(legs['mixed'][1], 'mixed', args.steps, args.warmup)
    res['mixed'] = (ms_val, ph_val, args.steps)
    k_side = max(1, min(args.steps, 2))
    for tag in [t for t in legs if t != 'mixed']:
        ks = k_side if tag == 'fp64' else 1
        ms, ph, _ = timed(legs[tag][1], tag, ks, 1)
        res[tag] = (ms, ph, ks)
    clocks = clk.stop()

    # block-row kernels alone (R = 8): FP64, FP32 and BF16 blocks of K, the
    # library's CUDA events around each launch, an L2 flush (256 MiB write)
    # between launches, after 2 warm-up launches
    o16 = o_of('bj', None, 0, 'fp32', 'restarted', 'bf16')
    driver.check(L.hdg_assemble(p.h, o16, st), 'assemble')       # builds the BF16 copy of K too
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    xv = torch.randn(p.n_dof * R, dtype=torch.float64, device=dev)
    yv = torch.empty_like(xv)
    pk = peaks()
    nnzb = nonzero_blocks(w)
    b = w.M * w.PF
    mv = {}
    for prec, name, sz, ld in ((0, 'fp64', 8, b), (1, 'fp32', 4, (b + 3) // 4 * 4), (2, 'bf16', 2, (b + 7) // 8 * 8)):
        for _ in range(2):
            driver.check(L.hdg_apply_K(p.h, prec, xv, yv, st), 'apply_K')
        torch.cuda.synchronize(dev)
        nrep = 10
        L.hdg_set_timing(p.h, 1)
        for _ in range(nrep):
            flush.fill_(1.0)
            driver.check(L.hdg_apply_K(p.h, prec, xv, yv, st), 'apply_K')
        torch.cuda.synchronize(dev)
        _, tms, nl = L.hdg_get_timing(p.h, prec)
        L.hdg_set_timing(p.h, 0)
        avg = tms / max(nl, 1)
        # algorithmic bytes: the real blocks (stored columns padded to 16 bytes
        # in FP32/BF16) + x read once + y written (FP64 x for FP64 blocks, its
        # FP32 copy otherwise)
        by = nnzb * b * ld * sz + p.n_dof * R * (16 if prec == 0 else 12)
        mv[name] = {'avg_ms': round(avg, 4), 'launches': int(nl), 'bytes_per_launch': int(by),
                    'gbs': round(by / avg / 1e6, 1), 'frac_hbm': round(by / avg / 1e6 / pk['hbm_gbs'], 3),
                    'tflops': round(2 * nnzb * b * b * R / avg / 1e9, 3),
                    'timing': 'CUDA events around each block-row launch, L2 flushed between launches'}

    # the dominant kernel inside the step: one more mixed step with the
    # library's per-launch events (launch by launch, no graphs), the FP32
    # block-row launches of K averaged
    driver.check(L.hdg_set_timing(p.h, 1), 'timing')
    step(legs['mixed'][1], 'mixed_timed', dvc, 1)
    torch.cuda.synchronize(dev)
    kp = 2 if args.poly_prec == 'bf16' else 1
    _, t32, n32 = L.hdg_get_timing(p.h, 1)
    _, t16, n16 = L.hdg_get_timing(p.h, 2)
    _, tbj, nbj = L.hdg_get_timing(p.h, 4)        # FP32 block-Jacobi applies of the polynomial
    L.hdg_set_timing(p.h, 0)
    # algorithmic bytes: the blocks, the FP32 x read, and the product written
    # in FP32 (the polynomial steps: 4 + 4 bytes per vector entry) or in FP64
    # and FP32 (the GMRES iteration's product: 4 + 8 + 4)
    its = infos.get('mixed_timed', infos.get('mixed', (0, 0, 0.0)))[0]
    blk32 = nnzb * b * ((b + 3) // 4 * 4) * 4
    blk16 = nnzb * b * ((b + 7) // 8 * 8) * 2
    by32 = blk32 + p.n_dof * R * 12
    by16 = blk16 + p.n_dof * R * 12
    it32 = min(its, n32) if not n16 else 0
    tot_by = (blk32 * n32 + p.n_dof * R * (16 * it32 + 8 * (n32 - it32)) +
              blk16 * n16 + p.n_dof * R * 8 * n16)
    tot_ms = t32 + t16
    achieved = tot_by / tot_ms / 1e6 if tot_ms > 0 else 0.0
    _, cfg32, _, _ = L.hdg_get_tuning(p.h, 0, 1)
    traffic, traffic_src = profiled_traffic(cfg32) if not n16 else (None, 'BF16 launches in the step')
    roof = {'kernel': 'blockrow_vec_kernel (face-block matvec y = K x, R = 8, FP32%s blocks, FP32 accumulation)'
                      % (' and BF16' if n16 else ''),
            'bound': 'hbm', 'achieved': round(achieved, 1), 'peak': pk['hbm_gbs'], 'unit': 'GB/s',
            'frac': round(achieved / pk['hbm_gbs'], 4), 'traffic': traffic, 'traffic_source': traffic_src,
            'bytes_per_launch': {'fp32_polynomial': int(blk32 + p.n_dof * R * 8),
                                 'fp32_iteration': int(blk32 + p.n_dof * R * 16), 'bf16': int(blk16 + p.n_dof * R * 8)},
            'launches_in_step': int(n32 + n16), 'ms_in_step': round(tot_ms, 3),
            'timing': 'CUDA events around every block-row launch of K in one mixed step run launch by launch',
            'peak_source': 'MEASURED_PEAKS.json hbm_gbs' if not pk.get('_fallback') else 'fallback 6.8 TB/s'}

    # the block-Jacobi applies of the same step: Chebyshev(4) is 5 applies per
    # preconditioner application, each reading the FP32 diagonal blocks
    # (stored columns padded to 16 bytes) and the FP32 input vector once;
    # their epilogues read and write the FP32 recurrence vectors r, d, z:
    # first apply writes 3 (16 bytes per entry with the input), the middle
    # ones read and write 3 (28), the last reads 3 and writes the FP64 result
    # (24)
    deg = 4
    pc_roof = None
    if nbj > 0 and nbj % (deg + 1) == 0:
        ents = p.n_dof * R
        bj_blocks = p.n_dof * ((b + 3) // 4 * 4) * 4
        by_app = (deg + 1) * bj_blocks + ents * (16 + 28 * (deg - 1) + 24)
        pc_ach = by_app * (nbj // (deg + 1)) / tbj / 1e6
        pc_roof = {'kernel': 'blockrow_vec_kernel (block-Jacobi apply z = D^-1 v, R = 8, FP32 blocks, Chebyshev '
                             'recurrence in the epilogue)',
                   'bound': 'hbm', 'achieved': round(pc_ach, 1), 'peak': pk['hbm_gbs'], 'unit': 'GB/s',
                   'frac': round(pc_ach / pk['hbm_gbs'], 4), 'bytes_per_application': int(by_app),
                   'launches_in_step': int(nbj), 'ms_in_step': round(tbj, 3),
                   'timing': 'CUDA events around every block-Jacobi launch of the polynomial in one mixed step '
                             'run launch by launch',
                   'peak_source': roof['peak_source']}

    # end to end through the C ABI from pinned host buffers: vertices, face
    # permutations, load vectors and Dirichlet values in; trace, u and q out
    e2e = None
    if not args.no_e2e:
        uh_host = torch.empty((w.n_face, w.M * w.PF, R), dtype=torch.float64).pin_memory()
        u_host = torch.empty((w.n_elem, w.M * w.PE, R), dtype=torch.float64).pin_memory()
        q_host = torch.empty((w.n_elem, w.M * w.D * w.PE, R), dtype=torch.float64).pin_memory()
        k_e2e = max(1, min(args.steps, 5))
        for _ in range(1):
            step(legs['mixed'][1], 'e2e', host, 0, outs=(uh_host, u_host, q_host))
        torch.cuda.synchronize(dev)
        if dist: dist.barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            step(legs['mixed'][1], 'e2e', host, 0, outs=(uh_host, u_host, q_host))
        torch.cuda.synchronize(dev)
        e_ms = (time.perf_counter() - t0) * 1e3 / k_e2e
        e_ms = max_over_ranks(e_ms, dist, dev)
        out_bytes = (uh_host.numel() + u_host.numel() + q_host.numel()) * 8
        e2e = {'value': round(e_ms, 3), 'unit': 'ms', 'h2d_bytes_per_step': int(in_bytes),
               'd2h_bytes_per_step': int(out_bytes), 'steps': k_e2e,
               'path': 'pinned host inputs (vertices, face permutations, load vectors, Dirichlet values) -> '
                       'hdg_condense_hex ... hdg_solve -> hdg_get_trace + hdg_recover into pinned host buffers'}
    p.close()
    del dvc
    torch.cuda.empty_cache()

    ms_mixed, ph_mixed, _ = res['mixed']
    ms_fp64, ph_fp64, k_fp64 = res['fp64']
    legs_out = {}
    for tag, (desc, _) in legs.items():
        ms, ph, ks = res[tag]
        it = infos.get(tag, (0, 0, 0.0))
        legs_out[tag] = {'solver': desc, 'ms_per_step': round(ms, 2), 'steps': ks,
                         'phases_ms': {k: round(v, 2) for k, v in ph.items()},
                         'gmres': it[0], 'refinement': it[1], 'rel_resid': it[2]}
    out = {
        'metric': METRIC, 'value': round(ms_mixed, 3), 'unit': 'ms', 'n_gpus': ws, 'steps': args.steps,
        'warmup': args.warmup, 'ms_per_step': round(ms_mixed, 3), 'higher_is_better': False, 'scaling': 'weak',
        'vs_baseline': None, 'dtype': 'f32 blocks / f64 Krylov', 'data': 'synthetic',
        'config': {'workload': WORKLOAD3 if n == 32 else WORKLOAD3.replace('32^3', '%d^3' % n),
                   'n_elem': w.n_elem, 'n_dof': p.n_dof, 'rhs': R, 'precond': 'block-Jacobi + Chebyshev(4)',
                   'restart': 50, 'rtol': 1e-8, 'solve': legs['mixed'][0],
                   'l2': 'inputs larger than L2 (FP32 K alone %.2f GB)' % (nnzb * b * ((b + 3) // 4 * 4) * 4 / 1e9),
                   'parallelism': 'replicas' if ws > 1 else 'single GPU'},
        'fp64_ms_per_step': round(ms_fp64, 3),
        'speedup_mixed_vs_fp64': round(ms_fp64 / ms_mixed, 3),
        'time_to_1e-8_solve_ms': {'mixed': round(ph_mixed['solve'], 2), 'fp64': round(ph_fp64['solve'], 2)},
        'speedup_mixed_vs_fp64_solve': round(ph_fp64['solve'] / ph_mixed['solve'], 3),
        'legs': legs_out,
        'block_matvec': mv,
        'autotuned': tuning,
        'roofline': roof,
        'precond_roofline': pc_roof,
        'gpu_launches': int(round(launches)),
        'clocks': clocks,
        'input_generation_s': round(t_in, 2),
    }
    if e2e:
        out['e2e'] = e2e
    if not args.no_config2:
        out['config2'] = config2_leg(args, local)
    if args.serving_requests > 0:
        out['serving'] = serving_leg(args, local)
    if rank == 0 and not args.no_cpu:
        out['cpu_baseline'] = cpu_baseline3(args)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return out


def config2_leg(args, local):
    """The 16^3 Q3 Poisson step (sin-product MMS, 1 RHS, BJ-GMRES(50) to
    1e-8, element blocks resident in HBM) with the plain FP64 solve and the
    preconditioner-only mixed solve (FP64 operator and Krylov, FP32 BJ
    inverses), min(steps, 5) timed steps each after 2 warm-up steps."""
    import numpy as np
    import torch
    from hdg_inputs import workloads as W
    from paper_2512_13619_gb300 import driver, _lib as L
    dev = torch.device('cuda', local)
    w = W.hex_poisson(n=16, k=3)
    blk = w.blocks()
    names = driver.BLOCK_NAMES
    dblk = {k: torch.from_numpy(np.ascontiguousarray(blk[k])).to(dev) for k in names}
    uD = torch.from_numpy(w.uhat_dirichlet()).to(dev)
    p = driver.Problem.from_workload(w, local)
    st = torch.cuda.current_stream(dev).cuda_stream
    u_dev = torch.empty((w.n_elem, w.M * w.PE, 1), dtype=torch.float64, device=dev)
    q_dev = torch.empty((w.n_elem, w.M * w.D * w.PE, 1), dtype=torch.float64, device=dev)
    opts = {'fp64': driver.opts(restart=50, rtol=1e-8, pc='bj', inner='fp64', max_iters=5000),
            'mixed_precond': driver.opts(restart=50, rtol=1e-8, pc='bj', inner='fp32', max_iters=5000, max_outer=-2),
            'mixed_restarted': driver.opts(restart=50, rtol=1e-8, pc='bj', inner='fp32', max_iters=5000,
                                           max_outer=-1)}
    out = {'workload': WORKLOAD, 'n_elem': w.n_elem, 'n_dof': p.n_dof}
    K = max(1, min(args.steps, 5))
    for tag, o in opts.items():
        def step():
            driver.check(L.hdg_condense(p.h, 0, w.n_elem, *[dblk[k] for k in names], 1, st), 'condense')
            driver.check(L.hdg_set_dirichlet(p.h, uD, 1, st), 'dirichlet')
            driver.check(L.hdg_assemble(p.h, o, st), 'assemble')
            driver.check(L.hdg_setup_precond(p.h, o, None, st), 'setup')
            info = L.hdg_solve_info()
            s_ = L.hdg_solve(p.h, o, st, info)
            if s_ != 0:
                raise RuntimeError('config2 %s: %s' % (tag, L.hdg_status_str(s_)))
            driver.check(L.hdg_recover(p.h, u_dev, q_dev, 1, st), 'recover')
            return info
        for _ in range(2):
            step()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(K):
            info = step()
        e1.record()
        torch.cuda.synchronize(dev)
        out[tag] = {'ms_per_step': round(e0.elapsed_time(e1) / K, 3), 'gmres': info.iters,
                    'rel_resid': info.rel_resid, 'steps': K}
    out['speedup_mixed_precond_vs_fp64'] = round(out['fp64']['ms_per_step'] / out['mixed_precond']['ms_per_step'], 3)
    p.close()
    del dblk
    torch.cuda.empty_cache()
    return out


def oracle_step3(w):
    """One step of the elasticity workload with the FP64 oracle: element
    blocks, condensation, assembly, block-Jacobi, Chebyshev(4) bounds from an
    Arnoldi(10) cycle on M^{-1} K, GMRES(50) to 1e-8 for every right-hand
    side, recovery.  Returns (ms, max iterations)."""
    import numpy as np
    from oracle.condense import condense_local
    from oracle.assemble import assemble, element_traces, recover
    from oracle import krylov, precond
    t0 = time.perf_counter()
    blk = w.blocks()
    uD = w.uhat_dirichlet()
    Kb, rb, rec = condense_local(blk, w.M, w.n_lfe)
    K, r = assemble(Kb, rb, w.mesh.elem_face, w.face_dirichlet, uD, w.M, w.PF)
    Binv = precond.bj_setup(K, w.M * w.PF)
    M = lambda v: precond.bj_apply(Binv, v)
    A = lambda v: M(K @ v)
    lo, hi = precond.chebyshev_bounds(A, w.random_vector(31), 10)
    Pinv = lambda v: precond.chebyshev_apply(A, lo, hi, 4, M(v))
    X = np.zeros_like(r)
    its = 0
    for c in range(w.R):
        X[:, c], info = krylov.gmres(lambda v: K @ v, Pinv, r[:, c], m=50, rtol=1e-8)
        its = max(its, info['iters'])
    ue = element_traces(X, w.mesh.elem_face, w.face_dirichlet, uD, w.M, w.PF)
    recover(rec, ue, w.M, w.n_lfe)
    return (time.perf_counter() - t0) * 1e3, its


def cpu_baseline3(args):
    from hdg_inputs import workloads as W
    w = W.hex_elasticity(n=ORACLE_SAMPLE_N, k=2, R=8)
    ms, it = oracle_step3(w)
    full = 32 ** 3
    return {'value': round(ms, 1), 'unit': 'ms', 'cores': cpu_cores(), 'kind': 'oracle',
            'sample': 'one full step of the same workload family on a %d^3 instance (%d of the %d elements, '
                      'seeded the same way): blocks, condensation, assembly, BJ + Chebyshev(4) set-up, GMRES(50) '
                      'to 1e-8 for all 8 RHS (%d iterations at most), recovery, FP64 on the host cores'
                      % (ORACLE_SAMPLE_N, w.n_elem, full, it),
            'per_element_ms': round(ms / w.n_elem, 3),
            'linear_extrapolation_to_32^3_ms': round(ms / w.n_elem * full, 1)}


def serving_leg(args, local):
    """The serving stream: HDG convection-diffusion requests (kappa
    log-uniform in [1e-3, 1], seeded unit velocity, n^3 hex meshes with n in
    8..24 and Q1..Q3) arriving as a seeded Poisson process; FP32 blocks with
    FP64 residuals at the restarts (restarted mixed mode), BJ-GMRES(30) to
    1e-8, admission by a device-memory budget.  Two schedulers: `lanes`
    (each request prepared and solved on its own lane's stream, GMRES cycles
    as CUDA graphs) and `batch` (lanes prepare, every prepared request is
    solved together in ONE persistent launch, hdg_solve_batch).  For each,
    the capacity is measured on a burst of the first requests, then the
    stream runs at 0.5x, 0.8x and 1.2x of it.  The meshes of the 51 shapes are
    generated before the stream starts (a request names a mesh the server
    holds); the element blocks of each request are computed from its kappa
    and velocity inside its latency."""
    import numpy as np
    from hdg_inputs import workloads as W
    from paper_2512_13619_gb300 import driver
    from paper_2512_13619_gb300.serving import HdgBackend, Server
    o = driver.opts(restart=30, rtol=1e-8, pc='bj', inner='fp32', inner_rtol=1e-4, max_iters=20000,
                    max_outer=-1 if args.serving_mixed == 'restarted' else 20)

    def inputs(shape, req):
        n, k = shape
        kappa, beta = (1.0, (1.0, 0.0, 0.0)) if req is None else (req['kappa'], req['beta'])
        return W.structured_convdiff_inputs(n, k, kappa, beta)

    reqs = W.serving_requests(args.serving_requests)
    for r in reqs:
        r['shape'] = (r['n'], r['k'])
    shapes = sorted({r['shape'] for r in reqs})
    probe = HdgBackend(inputs, o, device=local)
    t0 = time.perf_counter()
    for sh in shapes:
        probe.slot_bytes(sh)                           # generates and caches the mesh
    t_mesh = time.perf_counter() - t0
    budget = int(args.serving_budget_gb * (1 << 30))
    out = {'requests': len(reqs), 'lanes': args.lanes, 'budget_gb': args.serving_budget_gb,
           'mesh_generation_s': round(t_mesh, 2),
           'solve': 'FP32 blocks, BJ-GMRES(30) to 1e-8, mixed mode: ' + args.serving_mixed,
           'latency': 'arrival to trace in host memory (includes element-block generation on the host)'}
    modes = ('lanes', 'batch') if args.serving_mixed == 'restarted' else ('lanes',)
    for mode in modes:
        be = HdgBackend(inputs, o, device=local)
        be._mesh_cache = probe._mesh_cache
        srv = Server(be, lanes=args.lanes, mem_budget=budget, batch=(mode == 'batch'))
        warm = srv.warm(shapes) if args.serving_warm else 0
        ncal = min(32, len(reqs))
        cal = [dict(r, id=('cal', r['id'])) for r in reqs[:ncal]]
        st_cal = srv.run(cal, np.zeros(ncal))           # burst: capacity (and first slots)
        cap = st_cal['solves_per_s']
        res = {'capacity_burst_solves_per_s': round(cap, 2), 'warm_slots': warm, 'loads': {}}
        for fac in (0.5, 0.8, 1.2):
            tag = '%.1fx' % fac
            rq = [dict(r, id=(tag, r['id'])) for r in reqs]
            st = srv.run(rq, W.poisson_arrivals(len(rq), fac * cap))
            got = [srv.results[r['id']] for r in rq if r['id'] in srv.results]
            its = np.array([x['iters'] for x in got]) if got else np.zeros(1)
            res['loads'][tag] = {
                'arrival_rate_per_s': round(fac * cap, 2), 'completed': st['completed'], 'errors': st['errors'],
                'p50_ms': round(st['p50_ms'], 3), 'p99_ms': round(st['p99_ms'], 3),
                'mean_ms': round(st['mean_ms'], 3), 'solves_per_s': round(st['solves_per_s'], 2),
                'gmres_iters_mean': float(its.mean()), 'max_rel_resid': max([x['rel'] for x in got] + [0.0])}
            print('serving %s %s: %s' % (mode, tag, res['loads'][tag]), file=sys.stderr, flush=True)
        res.update({'slot_creations': srv.creations, 'evictions': srv.evictions,
                    'max_in_flight': srv.max_in_flight})
        if mode == 'batch':
            res['batches'] = srv.batches
            res['mean_batch'] = round(float(np.mean(srv.batch_sizes)), 2) if srv.batch_sizes else None
        srv.close()
        out[mode] = res
    return out


def run_config(args, local):
    """Solver and kernel measurements on a large problem: condensation,
    assembly, preconditioner set-up and GMRES to 1e-8 with the plain FP64
    path and the mixed path (FP32 blocks, FP64 refinement), per
    preconditioner; block-row products after autotuning (HBM GB/s)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from hdg_inputs import workloads as W
    from paper_2512_13619_gb300 import driver, _lib as L
    torch.cuda.set_device(local)
    dev = torch.device('cuda', local)
    names = driver.BLOCK_NAMES
    t_gen = time.perf_counter()
    nmesh = args.mesh_n or (40 if args.workload == 'cdr40' else 32)
    if args.workload == 'cdr40':
        w = W.hex_cdr(n=nmesh, k=2, R=4)
        hb, strides = W.shared_blocks(w)
        dblk = {k: torch.from_numpy(hb[k]).to(dev) for k in names}
        cases = [('bj', None, 0, 'fp32', 'fp32'), ('bj', 'gmres', 10, 'fp32', 'bf16')]
        desc = 'HDG 5-component CDR, %d^3 hex, Q2 (45 dofs/face, 270x270 element blocks), 4 RHS' % nmesh
    else:
        w = W.hex_elasticity(n=nmesh, k=2, R=8)
        dblk = {}
        sizes = None
        ch = 1024
        for c0 in range(0, w.n_elem, ch):
            b = w.blocks(c0, min(w.n_elem, c0 + ch))
            if sizes is None:
                dblk = {k: torch.empty((w.n_elem,) + b[k].shape[1:], dtype=torch.float64, device=dev) for k in names}
                sizes = True
            for k in names:
                dblk[k][c0:c0 + b[k].shape[0]].copy_(torch.from_numpy(np.ascontiguousarray(b[k])))
        strides = [dblk[k][0].numel() for k in names]
        cases = [('asm', None, 0, 'fp32', 'fp32'), ('bj', 'chebyshev', 4, 'fp32', 'fp32')]
        desc = 'HDG elasticity, %d^3 perturbed hex, Q2 (27 dofs/face, 162x162 element blocks), 8 RHS' % nmesh
    t_gen = time.perf_counter() - t_gen
    R = w.R
    st = torch.cuda.current_stream(dev).cuda_stream
    p = driver.Problem.from_workload(w, local)
    ptrs = [dblk[k] for k in names]

    def ev_time(fn, reps=1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    def condense():
        driver.check(L.hdg_condense_strided(p.h, 0, w.n_elem, ptrs, strides, 1, st), 'condense')
    condense()
    ms_cond = ev_time(condense)
    print('condensation %.1f ms' % ms_cond, file=sys.stderr, flush=True)
    cflops = condense_flops(w) * w.n_elem
    driver.check(L.hdg_set_dirichlet(p.h, w.uhat_dirichlet(), 0, st), 'dirichlet')
    out = {'workload': desc, 'n_elem': w.n_elem, 'n_dof': p.n_dof, 'rhs': R, 'input_generation_s': round(t_gen, 1),
           'condense_ms': round(ms_cond, 2), 'condense_tflops': round(cflops / ms_cond / 1e9, 3),
           'condense_frac_fp64_alu': round(cflops / ms_cond / 1e9 / FP64_ALU_PEAK_TFLOPS, 3), 'solves': []}
    pk = peaks()
    v0 = torch.from_numpy(w.random_vector(11)).to(dev)       # start vector of the polynomial's Arnoldi cycle
    for pc, poly, deg, inner, pprec in cases:
        row = {'pc': pc, 'poly': poly, 'degree': deg}
        for tag in ('fp64', 'mixed', 'mixed_restarted'):
            o = driver.opts(restart=50, rtol=1e-8, pc=pc, poly=poly, degree=deg,
                            inner='fp64' if tag == 'fp64' else inner, poly_prec='fp64' if tag == 'fp64' else pprec,
                            inner_rtol=1e-4, max_iters=args.max_iters,
                            max_outer=-1 if tag == 'mixed_restarted' else 20)
            ms_setup = ev_time(lambda: (driver.check(L.hdg_assemble(p.h, o, st), 'assemble'),
                                        driver.check(L.hdg_setup_precond(p.h, o, v0 if poly else None, st),
                                                     'setup')))
            info = L.hdg_solve_info()
            stt = L.hdg_solve(p.h, o, st, info)          # builds the cycle graphs
            print('%s %s %s: status %s, %d iterations, rel %.3g' % (pc, poly, tag, L.hdg_status_str(stt),
                                                                   info.iters, info.rel_resid),
                  file=sys.stderr, flush=True)
            if stt == 0:
                ms = ev_time(lambda: L.hdg_solve(p.h, o, st, info))
            else:
                ms = float('nan')
            row[tag] = {'setup_ms': round(ms_setup, 2), 'solve_ms': round(ms, 2), 'gmres': info.iters,
                        'refinement': info.outer, 'rel_resid': info.rel_resid, 'status': L.hdg_status_str(stt)}
        row['speedup_mixed_vs_fp64'] = round(row['fp64']['solve_ms'] / row['mixed']['solve_ms'], 3)
        row['speedup_mixed_restarted_vs_fp64'] = round(row['fp64']['solve_ms'] / row['mixed_restarted']['solve_ms'], 3)
        out['solves'].append(row)
        # block-row products after autotuning: K at every stored precision, the base preconditioner
        driver.check(L.hdg_autotune(p.h, 10, 0, st), 'autotune')
        fd = w.face_dirichlet
        nfree_e = (fd[w.mesh.elem_face] == 0).sum(axis=1)
        nnzb = int((nfree_e ** 2).sum() - w.n_free)
        b = w.M * w.PF
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
        xv = torch.randn(p.n_dof * R, dtype=torch.float64, device=dev)
        yv = torch.empty_like(xv)
        kern = {}
        for prec, pname, sz in ((0, 'fp64', 8), (1, 'fp32', 4), (2, 'bf16', 2)):
            if L.hdg_apply_K(p.h, prec, xv, yv, st) != 0:
                continue
            tot = 0.0
            for _ in range(5):
                flush.fill_(1.0)
                tot += ev_time(lambda: driver.check(L.hdg_apply_K(p.h, prec, xv, yv, st), 'apply_K'))
            avg = tot / 5
            by = nnzb * b * b * sz + p.n_dof * R * (16 if prec == 0 else 24)
            _, cfg, us, us0 = L.hdg_get_tuning(p.h, 0, prec)
            kern['K_' + pname] = {'avg_ms': round(avg, 4), 'gbs': round(by / avg / 1e6, 1),
                                  'frac_hbm': round(by / avg / 1e6 / pk['hbm_gbs'], 3), 'tuned_cfg': cfg,
                                  'tuned_us': round(us, 1), 'default_us': round(us0, 1)}
        op = 1 if pc == 'bj' else 2
        o = driver.opts(restart=50, pc=pc)
        for prec, pname in ((0, 'fp64'), (1, 'fp32')):
            _, cfg, us, us0 = L.hdg_get_tuning(p.h, op, prec)
            if us > 0:
                kern[pc + '_' + pname] = {'tuned_cfg': cfg, 'tuned_us': round(us, 1), 'default_us': round(us0, 1)}
        row['kernels'] = kern
    p.close()
    return out


def run_beam(args, local):
    """Sec. 6.2 cantilever beam (0,5) x (0,1) x (0,1), lambda = mu = 1,
    clamped at x = 0, uniform traction at x = 5: per mesh and degree, the
    condensation, the preconditioner set-up and GMRES(50) with classical
    Gram-Schmidt to a relative residual of 1e-6 (FP64), with BJ, BJ-PP(10),
    ASM and ASM-PP(10), timed with CUDA events; the polynomial variants also
    with the restarted mixed path (FP32 cycles, FP64 residual at restarts)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from hdg_inputs import workloads as W
    from paper_2512_13619_gb300 import driver, _lib as L
    torch.cuda.set_device(local)
    dev = torch.device('cuda', local)
    st = torch.cuda.current_stream(dev).cuda_stream
    names = driver.BLOCK_NAMES
    maxit = max(args.max_iters, 20000)

    def ev_time(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b)

    rows = []
    for case in args.beam_cases.split(','):
        n, k = (int(v) for v in case.split(':'))
        w = W.hex_beam(n=n, k=k)
        hb, strides = W.shared_blocks(w)
        dblk = [torch.from_numpy(hb[x]).to(dev) for x in names]
        p = driver.Problem.from_workload(w, local)

        def condense():
            driver.check(L.hdg_condense_strided(p.h, 0, w.n_elem, dblk, strides, 1, st), 'condense')
        condense()
        ms_cond = ev_time(condense)
        driver.check(L.hdg_set_dirichlet(p.h, w.uhat_dirichlet(), 0, st), 'dirichlet')
        v0 = torch.from_numpy(w.random_vector(11)).to(dev)
        row = {'N_E': w.n_elem, 'k': k, 'n_dof': p.n_dof, 'condense_ms': round(ms_cond, 3), 'solves': {}}
        for label, pc, poly in (('BJ', 'bj', None), ('BJ-PP(10)', 'bj', 'gmres'), ('ASM', 'asm', None),
                                ('ASM-PP(10)', 'asm', 'gmres')):
            for tag in (('fp64', 'mixed_restarted') if poly else ('fp64',)):
                o = driver.opts(restart=50, rtol=1e-6, orth='cgs', pc=pc, poly=poly, degree=10 if poly else 0,
                                inner='fp64' if tag == 'fp64' else 'fp32',
                                poly_prec='fp64' if tag == 'fp64' else 'fp32', max_iters=maxit,
                                max_outer=-1 if tag != 'fp64' else 20)
                ms_setup = ev_time(lambda: (driver.check(L.hdg_assemble(p.h, o, st), 'assemble'),
                                            driver.check(L.hdg_setup_precond(p.h, o, v0 if poly else None, st),
                                                         'setup')))
                info = L.hdg_solve_info()
                stt = L.hdg_solve(p.h, o, st, info)          # builds the cycle graphs
                ms = ev_time(lambda: L.hdg_solve(p.h, o, st, info)) if stt == 0 else float('nan')
                print('beam N_E=%d k=%d %s %s: %s, %d iterations, %.2f ms' % (
                    w.n_elem, k, label, tag, L.hdg_status_str(stt), info.iters, ms), file=sys.stderr, flush=True)
                row['solves'][label + ('' if tag == 'fp64' else ' mixed')] = {
                    'gmres': info.iters, 'setup_ms': round(ms_setup, 3), 'solve_ms': round(ms, 3),
                    't_comp_s': round((ms_cond + ms_setup + ms) / 1e3, 4), 'rel_resid': info.rel_resid,
                    'status': L.hdg_status_str(stt)}
        # mean tip deflection of the last solution: <g, uhat> over the loaded
        # face (unit area, t = (0, 0, -1)), from the element face loads r_uh
        # (identical face parametrisation from both sides on this mesh)
        tr = p.trace()[:, :, 0]
        ruh = hb['ruh'][:, :, 0].reshape(w.n_elem, w.n_lfe, -1)
        row['tip_deflection'] = round(float(np.einsum('elj,elj->', ruh, tr[w.mesh.elem_face])), 4)
        rows.append(row)
        p.close()
        del dblk
        torch.cuda.empty_cache()
    return {'workload': 'HDG linear elasticity cantilever beam (0,5)x(0,1)^2, lambda = mu = 1, Q^k hexahedra, '
                        'clamped x = 0, traction (0,0,-1) at x = 5; GMRES(50) CGS to 1e-6',
            'data': 'synthetic', 'max_iters': maxit, 'cases': rows}


def run_beamcheck(args, local):
    """The Sec. 6.2 beam at N_E = 1080, k = 3 (5n x n x n with n = 6, or
    --mesh-n): the harmonic Ritz values of the BJ-PP(10) set-up on the GPU
    against the oracle's (Arnoldi(10) with MGS on BJ^{-1} K from the same
    start vector, on the host), and the GPU's BJ-PP(10) GMRES(50)-CGS
    iteration counts to 1e-6 from three seeded start vectors."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from hdg_inputs import workloads as W
    from paper_2512_13619_gb300 import driver, _lib as L
    from oracle import precond
    from oracle.condense import condense_local
    from oracle.assemble import assemble
    torch.cuda.set_device(local)
    dev = torch.device('cuda', local)
    st = torch.cuda.current_stream(dev).cuda_stream
    n = args.mesh_n or 6
    w = W.hex_beam(n=n, k=3)
    hb, strides = W.shared_blocks(w)
    p = driver.Problem.from_workload(w, local)
    dblk = [torch.from_numpy(hb[x]).to(dev) for x in driver.BLOCK_NAMES]
    driver.check(L.hdg_condense_strided(p.h, 0, w.n_elem, dblk, strides, 1, st), 'condense')
    driver.check(L.hdg_set_dirichlet(p.h, w.uhat_dirichlet(), 0, st), 'dirichlet')
    t0 = time.perf_counter()
    full = {k: np.repeat(hb[k], w.n_elem, axis=0) if strides[i] == 0 else hb[k]
            for i, k in enumerate(driver.BLOCK_NAMES)}
    Kb, rb, _ = condense_local(full, w.M, w.n_lfe)
    K, r = assemble(Kb, rb, w.mesh.elem_face, w.face_dirichlet, w.uhat_dirichlet(), w.M, w.PF)
    Binv = precond.bj_setup(K, w.M * w.PF)
    A = lambda v: precond.bj_apply(Binv, K @ v)
    t_or = time.perf_counter() - t0
    rows = []
    for seed in (11, 12, 13):
        v0 = w.random_vector(seed)
        o = driver.opts(restart=50, rtol=1e-6, orth='cgs', pc='bj', poly='gmres', degree=10, max_iters=20000)
        p.assemble(o)
        p.setup_precond(o, v0)
        th_gpu = p.poly()
        th_or = precond.pp_setup(A, v0, 10)
        key = lambda t: (round(t.real, 9), round(t.imag, 9))
        a, b = sorted(th_gpu, key=key), sorted(th_or, key=key)
        dev_rel = float(max(abs(x - y) for x, y in zip(a, b)) / max(abs(y) for y in b)) if len(a) == len(b) else None
        stt, info = p.solve(o)
        rows.append({'seed': seed, 'gmres': info.iters, 'status': L.hdg_status_str(stt), 'rel_resid': info.rel_resid,
                     'ritz_count_gpu': len(th_gpu), 'ritz_count_oracle': len(th_or),
                     'ritz_max_rel_diff': dev_rel, 'min_abs_ritz': float(min(abs(th_or))),
                     'max_abs_ritz': float(max(abs(th_or)))})
        print('beamcheck seed %d: %s' % (seed, rows[-1]), file=sys.stderr, flush=True)
    p.close()
    return {'workload': 'Sec. 6.2 beam, N_E = %d, Q3, BJ-PP(10) GMRES(50)-CGS to 1e-6' % w.n_elem,
            'n_dof': int(K.shape[0]), 'oracle_setup_s': round(t_or, 1), 'seeds': rows}


def run_tets(args, local):
    """Sec. 6.1 three-dimensional Poisson runs, synthetic stand-in: Laplace on
    (-1,1)^3 minus a central cube (u = 0 there, outward flux n_x on the box),
    Kuhn tetrahedra, P^k; BJ-PP(10), BJ-PP(20), ASM-PP(10), ASM-PP(20) with
    GMRES(50)-CGS to 1e-6 in FP64, set-up and solve timed with CUDA events."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from hdg_inputs import workloads as W
    from paper_2512_13619_gb300 import driver, _lib as L
    torch.cuda.set_device(local)
    dev = torch.device('cuda', local)
    st = torch.cuda.current_stream(dev).cuda_stream
    n = args.mesh_n or 26
    names9 = driver.BLOCK_NAMES[:9]

    def ev_time(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b)

    rows = []
    for k in [int(v) for v in args.tet_ks.split(',')]:
        t_gen = time.perf_counter()
        w = W.tet_obstacle(n=n, k=k)
        rb, cls, ruh = W.class_blocks(w)
        t_gen = time.perf_counter() - t_gen
        p = driver.Problem.from_workload(w, local)
        t0 = time.perf_counter()
        ch = 8192
        for c0 in range(0, w.n_elem, ch):
            c1 = min(w.n_elem, c0 + ch)
            b = {x: np.ascontiguousarray(rb[x][cls[c0:c1]]) for x in names9}
            b['ru'] = np.zeros((c1 - c0, w.M * w.PE, 1))
            b['ruh'] = np.ascontiguousarray(ruh[c0:c1])
            p.condense(b, c0)
        torch.cuda.synchronize(dev)
        t_cond = time.perf_counter() - t0
        driver.check(L.hdg_set_dirichlet(p.h, w.uhat_dirichlet(), 0, st), 'dirichlet')
        v0 = torch.from_numpy(w.random_vector(11)).to(dev)
        row = {'N_E': w.n_elem, 'k': k, 'n_dof': p.n_dof, 'input_generation_s': round(t_gen, 1),
               'condense_from_host_s': round(t_cond, 2), 'solves': {}}
        for label, pc, deg in (('BJ-PP(10)', 'bj', 10), ('BJ-PP(20)', 'bj', 20), ('ASM-PP(10)', 'asm', 10),
                               ('ASM-PP(20)', 'asm', 20)):
            o = driver.opts(restart=50, rtol=1e-6, orth='cgs', pc=pc, poly='gmres', degree=deg,
                            poly_prec='fp64', max_iters=max(args.max_iters, 3000))
            ms_setup = ev_time(lambda: (driver.check(L.hdg_assemble(p.h, o, st), 'assemble'),
                                        driver.check(L.hdg_setup_precond(p.h, o, v0, st), 'setup')))
            info = L.hdg_solve_info()
            stt = L.hdg_solve(p.h, o, st, info)
            ms = ev_time(lambda: L.hdg_solve(p.h, o, st, info)) if stt == 0 else float('nan')
            print('tets N_E=%d k=%d %s: %s, %d iterations, %.2f ms' % (w.n_elem, k, label, L.hdg_status_str(stt),
                                                                     info.iters, ms), file=sys.stderr, flush=True)
            row['solves'][label] = {'gmres': info.iters, 'setup_ms': round(ms_setup, 3), 'solve_ms': round(ms, 3),
                                    'rel_resid': info.rel_resid, 'status': L.hdg_status_str(stt)}
        rows.append(row)
        p.close()
        torch.cuda.empty_cache()
    return {'workload': 'HDG Poisson (Laplace) on (-1,1)^3 minus a central cube of half-width 0.25, Kuhn '
                        'tetrahedra, P^k; u = 0 on the obstacle, outward flux n_x on the box; GMRES(50) CGS to 1e-6',
            'data': 'synthetic', 'cases': rows}


def run_burgers(args, local):
    """Sec. 6.1 steady viscous Burgers problem (nu = 1/200, u = 1 - 2x on three
    sides, outflow at y = 1) on (1/h)^2 Q^k quadrilaterals: damped Newton to a
    residual of 1e-8 from u = 1 - 2x, each step's linear solve GMRES(50)-CGS
    to 1e-6 with BJ, BJ-PP(10), ASM or ASM-PP(10) on the GPU; the total
    GMRES iterations over the Newton steps, and the time spent in the
    library's calls and in the host's residual and Jacobian evaluations."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from hdg_inputs import burgers as BG
    from paper_2512_13619_gb300 import driver
    from paper_2512_13619_gb300.newton import newton_solve
    torch.cuda.set_device(local)
    rows = []
    for case in args.burgers_cases.split(','):
        k, n = (int(v) for v in case.split(':'))
        P = BG.Burgers(n=n, k=k)
        v0 = np.random.default_rng(11).standard_normal(P.n_free * P.PF)
        row = {'k': k, '1/h': n, 'n_dof': P.n_free * P.PF, 'solves': {}}
        for label, pc, deg in (('BJ', 'bj', 0), ('BJ-PP(10)', 'bj', 10), ('ASM', 'asm', 0), ('ASM-PP(10)', 'asm', 10)):
            o = driver.opts(restart=50, rtol=1e-6, orth='cgs', pc=pc, poly='gmres' if deg else None, degree=deg,
                            poly_prec='fp64', max_iters=max(args.max_iters, 20000))
            try:
                _, info = newton_solve(P, o, v0 if deg else None, tol=1e-8, device=local)
                h = info['history']
                rec = {'newton_steps': len(h) - 1, 'gmres': info['gmres'], 'final_residual': h[-1][0],
                       'linear_s': round(info['linear_s'], 3), 'host_s': round(info['host_s'], 3),
                       'status': 'ok' if h[-1][0] <= 1e-8 else 'newton not converged'}
            except RuntimeError as e:
                rec = {'status': str(e)}
            print('burgers k=%d 1/h=%d %s: %s' % (k, n, label, rec), file=sys.stderr, flush=True)
            row['solves'][label] = rec
        rows.append(row)
    return {'workload': 'HDG steady viscous Burgers u_y + (u^2/2)_x - (1/200) lap u = 0 on (0,1)^2, Q^k '
                        'quadrilaterals, tau = 2; damped Newton to 1e-8, GMRES(50) CGS to 1e-6 per step',
            'data': 'synthetic', 'cases': rows}


def oracle_step(w, blk):
    """One step of the workload with the FP64 oracle (condense, assemble,
    block-Jacobi, GMRES(50) to 1e-8, recover).  Returns (ms, iterations)."""
    from oracle.condense import condense_local
    from oracle.assemble import assemble, element_traces, recover
    from oracle import krylov, precond
    t0 = time.perf_counter()
    uD = w.uhat_dirichlet()
    Kb, rb, rec = condense_local(blk, w.M, w.n_lfe)
    K, r = assemble(Kb, rb, w.mesh.elem_face, w.face_dirichlet, uD, w.M, w.PF)
    Binv = precond.bj_setup(K, w.M * w.PF)
    x, info = krylov.gmres(lambda v: K @ v, lambda v: precond.bj_apply(Binv, v), r[:, 0], m=50, rtol=1e-8)
    ue = element_traces(x[:, None], w.mesh.elem_face, w.face_dirichlet, uD, w.M, w.PF)
    recover(rec, ue, w.M, w.n_lfe)
    return (time.perf_counter() - t0) * 1e3, info['iters']


def cpu_cores():
    try:
        import numpy  # noqa: F401
        from threadpoolctl import threadpool_info
        n = max([i.get('num_threads', 1) for i in threadpool_info()] + [1])
        return n
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(args, w, blk):
    ms, it = oracle_step(w, blk)
    return {'value': round(ms, 1), 'unit': 'ms', 'cores': cpu_cores(), 'kind': 'oracle',
            'sample': 'one full step of the same workload (condense all %d elements, assemble, BJ setup, '
                      'BJ-GMRES(50) to 1e-8 in FP64: %d iterations, recover) on the host cores' % (w.n_elem, it)}


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    if args.workload == 'step3':
        return run_reference3(args, ws)
    from hdg_inputs import workloads as W
    w = W.hex_poisson(n=args.n, k=args.k)
    blk = w.blocks()
    for _ in range(args.warmup):
        oracle_step(w, blk)
    ts = []
    for _ in range(args.steps):
        ts.append(oracle_step(w, blk)[0])
    ms = sum(ts) / len(ts)
    cores = cpu_cores()
    return {'impl': 'reference', 'metric': METRIC, 'value': round(ms, 1), 'unit': 'ms', 'n_gpus': ws,
            'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': round(ms, 1), 'higher_is_better': False,
            'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic',
            'config': {'workload': WORKLOAD, 'n_elem': w.n_elem, 'n_dof': w.n_dof, 'precond': 'block-Jacobi',
                       'restart': 50, 'rtol': 1e-8, 'rhs': w.R, 'solve': 'FP64 oracle (CPU)',
                       'parallelism': 'rank 0 only'},
            'cpu_baseline': {'value': round(ms, 1), 'unit': 'ms', 'cores': cores, 'kind': 'oracle',
                             'sample': 'full steps of the workload with the FP64 CPU oracle'},
            'e2e': {'value': round(ms, 1), 'unit': 'ms', 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0}}


def run_reference3(args, ws):
    """The oracle arm of the default step: each step is the FP64 oracle's
    full step on the bounded 6^3 sample of the elasticity workload."""
    from hdg_inputs import workloads as W
    w = W.hex_elasticity(n=ORACLE_SAMPLE_N, k=2, R=8)
    for _ in range(args.warmup):
        oracle_step3(w)
    ts, it = [], 0
    for _ in range(args.steps):
        ms, it = oracle_step3(w)
        ts.append(ms)
    ms = sum(ts) / len(ts)
    cores = cpu_cores()
    sample = ('each step: the FP64 oracle (blocks, condensation, assembly, BJ + Chebyshev(4), GMRES(50) to 1e-8 for '
              '8 RHS, recovery) on a %d^3 instance of the workload (%d elements, %d iterations at most)'
              % (ORACLE_SAMPLE_N, w.n_elem, it))
    return {'impl': 'reference', 'metric': METRIC, 'value': round(ms, 1), 'unit': 'ms', 'n_gpus': ws,
            'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': round(ms, 1), 'higher_is_better': False,
            'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic',
            'config': {'workload': WORKLOAD3, 'n_elem': 32 ** 3, 'rhs': 8, 'precond': 'block-Jacobi + Chebyshev(4)',
                       'restart': 50, 'rtol': 1e-8, 'solve': 'FP64 oracle (CPU), bounded sample',
                       'sample_n_elem': w.n_elem, 'parallelism': 'rank 0 only'},
            'cpu_baseline': {'value': round(ms, 1), 'unit': 'ms', 'cores': cores, 'kind': 'oracle', 'sample': sample},
            'e2e': {'value': round(ms, 1), 'unit': 'ms', 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0}}


def run_profile(args):
    """Minimal set-up for a profiler: the workload on cuda:0, then the
    kernels under study once."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from hdg_inputs import workloads as W
    from paper_2512_13619_gb300 import driver, _lib as L
    if args.profile in ('step3', 'matvec3'):
        w = W.hex_elasticity(n=args.mesh_n or 32, k=2, R=8)
        verts, perm, nquad = driver.hex_geometry_inputs(w)
        ru, ruh = w.load_vectors()
        d = {k: torch.from_numpy(v).cuda() for k, v in (('verts', verts), ('perm', perm), ('ru', ru), ('ruh', ruh))}
        phys, _keep = L.physics(w.phys.Cq, w.phys.Cu, w.phys.Rr, w.phys.tau)
        v0 = w.random_vector(31)
        mo = {'restarted': -1, 'refinement': 20, 'precond': -2}[args.mixed_mode]
        o = driver.opts(restart=50, rtol=1e-8, pc='bj', poly='chebyshev', degree=4, inner='fp32',
                        poly_prec=args.poly_prec, inner_rtol=1e-4, max_iters=3000, max_outer=mo)
        p = driver.Problem.from_workload(w, 0)
        if args.no_graphs:
            L.hdg_set_graphs(p.h, 0)
        if args.profile == 'matvec3':
            driver.check(L.hdg_condense_hex(p.h, 0, w.n_elem, nquad, d['verts'], d['perm'], phys, d['ru'], d['ruh'],
                                            1), 'condense_hex')
            p.set_dirichlet(np.zeros((w.n_face, w.M * w.PF, w.R)))
            o16 = driver.opts(pc='bj', inner='fp32', poly_prec='bf16')
            p.assemble(o16)
            p.setup_precond(o16)
            driver.check(L.hdg_autotune(p.h, 5, 0, None), 'autotune')
            if args.k32_config:
                # the FP32 product in a given launch configuration (kind, slot
                # parts, CTAs per SM), e.g. the one tuned at another mesh size
                cfg = [int(v) for v in args.k32_config.split(',')]
                driver.check(L.hdg_set_tuning(p.h, 0, L.HDG_FP32, cfg), 'set_tuning')
            x = torch.randn(p.n_dof * w.R, dtype=torch.float64, device='cuda')
            y = torch.empty_like(x)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push('matvec')
            for prec in (L.HDG_FP64, L.HDG_FP32, L.HDG_BF16):
                driver.check(L.hdg_apply_K(p.h, prec, x, y), 'apply_K')
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
            p.close()
            print('profile run done')
            return
        for it in range(2):
            if it == 1:
                torch.cuda.synchronize()
                torch.cuda.nvtx.range_push('step2')        # the whole second step
            driver.check(L.hdg_condense_hex(p.h, 0, w.n_elem, nquad, d['verts'], d['perm'], phys, d['ru'], d['ruh'],
                                            1), 'condense_hex')
            p.set_dirichlet(np.zeros((w.n_face, w.M * w.PF, w.R)))
            p.assemble(o)
            p.setup_precond(o, v0)
            if it == 0:
                driver.check(L.hdg_autotune(p.h, 10, 0, None), 'autotune')
            else:
                torch.cuda.nvtx.range_push('solve2')       # the second solve, for range-filtered captures
            st, info = p.solve(o)
            if it == 1:
                torch.cuda.synchronize()
                torch.cuda.nvtx.range_pop()
            driver.check(st, 'solve')
            p.recover()
            if it == 1:
                torch.cuda.synchronize()
                torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        print('iterations', info.iters)
        p.close()
        print('profile run done')
        return
    w = W.hex_poisson(n=args.n, k=args.k)
    p = driver.Problem.from_workload(w, 0)
    if args.profile == 'generate':
        verts, perm, nquad = driver.hex_geometry_inputs(w)
        dv, dp = torch.from_numpy(verts).cuda(), torch.from_numpy(perm).cuda()
        phys, _keep = L.physics(w.phys.Cq, w.phys.Cu, w.phys.Rr, w.phys.tau)
        one = w.blocks(0, 1)
        out = [torch.empty((w.n_elem,) + one[k].shape[1:], dtype=torch.float64, device='cuda')
               for k in driver.BLOCK_NAMES[:9]]
        for _ in range(2):
            driver.check(L.hdg_hex_blocks(p.h, w.n_elem, nquad, dv, dp, phys, out, 1), 'hex_blocks')
        torch.cuda.synchronize()
        p.close()
        print('profile run done')
        return
    blk = w.blocks()
    if args.no_graphs:
        L.hdg_set_graphs(p.h, 0)
    dblk = {k: torch.from_numpy(np.ascontiguousarray(blk[k])).cuda() for k in driver.BLOCK_NAMES}
    p.condense(dblk, 0, on_device=True)
    if args.profile == 'matvec':
        o = driver.opts(pc='bj')
        p.set_dirichlet(w.uhat_dirichlet())
        p.assemble(o)
        x = torch.randn(p.n_dof * w.R, dtype=torch.float64, device='cuda')
        y = torch.empty_like(x)
        for prec in (L.HDG_FP64, L.HDG_FP32):
            driver.check(L.hdg_apply_K(p.h, prec, x, y), 'apply_K')
    elif args.profile.startswith('solve'):
        inner = 'fp32' if args.profile == 'solve-mixed' else 'fp64'
        o = driver.opts(restart=50, rtol=1e-8, pc='bj', inner=inner, inner_rtol=1e-4, max_iters=5000)
        p.set_dirichlet(w.uhat_dirichlet())
        p.assemble(o)
        p.setup_precond(o)
        for _ in range(2):      # the first solve builds the cycle graphs
            st, info = p.solve(o)
            driver.check(st, 'solve')
        print('iterations', info.iters, 'refinement', info.outer)
    torch.cuda.synchronize()
    p.close()
    print('profile run done')


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.profile:
        run_profile(args)
        return
    if args.impl == 'reference':
        out = run_reference(args, ws, rank)
    elif args.workload == 'beam':
        out = run_beam(args, local)
    elif args.workload == 'beamcheck':
        out = run_beamcheck(args, local)
    elif args.workload == 'tets':
        out = run_tets(args, local)
    elif args.workload == 'burgers':
        out = run_burgers(args, local)
    elif args.workload == 'step3':
        out = run_step3(args, ws, rank, local)
    elif args.workload != 'poisson16':
        out = run_config(args, local)
    else:
        out = run_ours(args, ws, rank, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == '__main__':
    main()
