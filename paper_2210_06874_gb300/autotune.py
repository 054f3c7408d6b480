"""Autotuner for the launch shape of the mixed-precision path.

For one chain it times short mixed CG solves with a fixed iteration count
(max_iter iterations, convergence not required: the per-iteration cost does
not depend on the residual) for candidate shapes -- CTAs of the persistent
launch (team_ctas), CTAs of the FP32 inner loop (inner_ctas), time slices per
tensor-core tile (tile_slices), streamed or resident E, site-major or
slice-major tiles, CUDA-core cluster mode, split-K tiles with E resident
(operand_mode) -- and keeps the fastest.  Timing uses CUDA
events on the current stream around calls through the C ABI; results are
cached per (L, Nt, team constraint) for the process.
"""
import itertools

import torch

from . import hmc

_cache = {}


def small_feasible(V, Nt, C):
    """Host copy of the feasibility rule of the CUDA-core cluster mode
    (operand_mode 3): 1 <= C <= 16 CTAs, each with 1..16 time slices, and the
    shared-memory layout within the 208 KB operand area."""
    if C < 1 or C > 16 or Nt < C or -(-Nt // C) > 16:
        return False
    S = -(-Nt // C)
    Vr = -(-V // 32) * 32
    SP = 2 if S <= 2 else 4 if S <= 4 else 8 if S <= 8 else 16
    G = Vr // 32
    KS = min(1 if G >= 8 else 8 // G, V)
    r16 = lambda b: (b + 15) // 16 * 16
    total = (r16(V * Vr * 4) + 6 * r16(S * V * 8) + 2 * r16(V * SP * 8) + 2 * r16(V * 8) +
             r16(KS * S * Vr * 8))
    return total <= 208 * 1024


def team_candidates(params, csize):
    """Shapes for a chain run as a thread-block-cluster team of csize CTAs
    (a batch's team chains): every CTA in the inner team; slice-major tiles
    (slices chosen by the library), site-major tiles of 8 or 16 slices, and
    the CUDA-core cluster mode where the chain fits it."""
    out = [(csize, csize, 0, 4), (csize, csize, 8, 1), (csize, csize, 16, 1)]
    if small_feasible(params.V, params.Nt, csize):
        out.append((csize, csize, 8, 3))
    return sorted(set(out))


def candidates(params, num_sms, single_cta=False):
    """Shapes (team_ctas, inner_ctas, tile_slices, operand_mode) worth timing:
    streamed E with one CTA or teams sized to the tensor-core / FP64 tile
    counts, resident E (one CTA per 128-site block) where E fits, the
    CUDA-core cluster mode (clusters of 1, 2, 4, 8 or 16 CTAs) where it fits
    (16 is a non-portable cluster size that a device may refuse; the tuner
    then skips it), and slice-major tiles (operand_mode 4, slices per tile
    chosen by the library: tile_slices 0) on one CTA or inner teams of 2, 4
    and 8 CTAs."""
    V, Nt = params.V, params.Nt
    nti = (V + 127) // 128
    vp = ((V + 63) // 64) * 64
    f64_tiles = ((V + 31) // 32) * ((Nt + 7) // 8)
    out = []
    for C in (1, 2, 4, 8, 16):
        if single_cta and C > 1:
            break
        if small_feasible(V, Nt, C):
            teams = {C} if single_cta else {C, max(C, min(f64_tiles, num_sms) // C * C)}
            for team in sorted(teams):
                out.append((team, C, 8, 3))
    for ns in (8, 16, 32):
        tiles = nti * ((Nt + ns - 1) // ns)
        if single_cta:
            out.append((1, 1, ns, 1))
            if vp <= 256 and nti == 1 and ns <= 16:
                out.append((1, 1, ns, 2))
            continue
        for inner in sorted({1, min(tiles, num_sms)}):
            for team in sorted({max(inner, min(f64_tiles, num_sms)), min(num_sms, max(inner, 1))}):
                out.append((team, inner, ns, 1))
        if vp <= 256 and nti <= num_sms and ns <= 16:
            out.append((max(nti, min(f64_tiles, num_sms)), nti, ns, 2))
    if single_cta:
        out.append((1, 1, 0, 4))
    else:
        for inner in (1, 2, 4, 8):
            out.append((max(inner, min(f64_tiles, num_sms)), inner, 0, 4))
        if V >= 128:
            # split-K tiles with E resident, clusters of C CTAs (the launch
            # takes as many clusters as fit; shapes the library refuses are
            # skipped); n-groups of the default size (at most 64 slices) or
            # of 32 or 16 slices (more clusters share a small lattice)
            for ns in (0, 32, 16):
                if ns and ns >= Nt:
                    continue
                for C in (2, 4, 6, 8):
                    out.append((0, C, ns, 5))
    return sorted(set(out))


def pick(timings):
    """(shape, seconds per iteration) pairs -> fastest shape (ties: fewer CTAs)."""
    return min(timings, key=lambda kv: (kv[1],) + tuple(kv[0]))[0]


def tune(params, iters=40, reps=2, single_cta=False, seed=1, team=0, modes=None):
    """Return a copy of params with team_ctas, inner_ctas, tile_slices and
    operand_mode set to the fastest measured shape (team > 1: among the
    shapes of a cluster team of that many CTAs; modes: only those operand
    modes, e.g. (5,) for mass preconditioning on the mixed path)."""
    key = (params.L, params.Nt, round(params.beta / params.Nt, 12), single_cta, team,
           tuple(modes) if modes else None)
    if key in _cache:
        (team_c, inner, ns, mode), _ = _cache[key]
    else:
        dev = torch.device("cuda", torch.cuda.current_device())
        num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
        g = torch.Generator(device="cpu").manual_seed(seed)
        V, Nt = params.V, params.Nt
        phi = (0.3 * torch.randn(Nt, V, generator=g, dtype=torch.float64)).to(dev)
        chi = torch.complex(torch.randn(Nt, V, generator=g, dtype=torch.float64),
                            torch.randn(Nt, V, generator=g, dtype=torch.float64)).to(dev)
        timings = []
        shapes = team_candidates(params, team) if team > 1 else candidates(params, num_sms,
                                                                             single_cta)
        if modes:
            shapes = [sh for sh in shapes if sh[3] in modes]
        for team_c, inner, ns, mode in shapes:
            p = hmc.Params(**{**params.__dict__, "team_ctas": team_c, "inner_ctas": inner,
                              "tile_slices": ns, "operand_mode": mode,
                              "precision": hmc.PREC_MIXED})
            ctx = hmc.Context(p)
            try:
                ctx.cg_solve(phi, chi, tol=1e-30, max_iter=4, prec=hmc.PREC_MIXED,
                             allow_not_converged=True)
            except hmc.HmcError:
                # a launch configuration this device (or a profiler) refuses
                ctx.close()
                continue
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            stream = torch.cuda.current_stream()
            s.record(stream)
            for _ in range(reps):
                ctx.cg_solve(phi, chi, tol=1e-30, max_iter=iters, prec=hmc.PREC_MIXED,
                             allow_not_converged=True)
            e.record(stream)
            e.synchronize()
            timings.append(((team_c, inner, ns, mode),
                            s.elapsed_time(e) * 1e-3 / (reps * iters)))
            ctx.close()
        best = pick(timings)
        _cache[key] = (best, dict(timings)[best])
        team_c, inner, ns, mode = best
    return hmc.Params(**{**params.__dict__, "team_ctas": team_c, "inner_ctas": inner,
                         "tile_slices": ns, "operand_mode": mode})


_ru_cache = {}


def tune_ru(params, candidates=(0.003, 0.01, 0.05, 0.2), seed=2):
    """Return a copy of params with the reliable-update threshold ru_delta
    that solves fastest to params.cg_tol, timed with full mixed solves in
    the params' launch shape (the best value depends on the chain: fewer
    FP64 updates pay where the FP64 work runs on few CTAs, frequent ones
    where the FP32 iteration stalls early)."""
    key = (params.L, params.Nt, round(params.beta / params.Nt, 12), params.team_ctas,
           params.inner_ctas, params.tile_slices, params.operand_mode, params.cg_tol)
    if key not in _ru_cache:
        dev = torch.device("cuda", torch.cuda.current_device())
        g = torch.Generator(device="cpu").manual_seed(seed)
        V, Nt = params.V, params.Nt
        phi = (0.3 * torch.randn(Nt, V, generator=g, dtype=torch.float64)).to(dev)
        chi = torch.complex(torch.randn(Nt, V, generator=g, dtype=torch.float64),
                            torch.randn(Nt, V, generator=g, dtype=torch.float64)).to(dev)
        timings = []
        for ru in candidates:
            ctx = hmc.Context(hmc.Params(**{**params.__dict__, "ru_delta": ru,
                                            "precision": hmc.PREC_MIXED}))
            try:
                ctx.cg_solve(phi, chi, tol=params.cg_tol, prec=hmc.PREC_MIXED)
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                stream = torch.cuda.current_stream()
                s.record(stream)
                ctx.cg_solve(phi, chi, tol=params.cg_tol, prec=hmc.PREC_MIXED)
                e.record(stream)
                e.synchronize()
                timings.append((ru, s.elapsed_time(e)))
            except hmc.HmcError:
                pass
            ctx.close()
        _ru_cache[key] = min(timings, key=lambda kv: kv[1])[0] if timings else 0.0
    return hmc.Params(**{**params.__dict__, "ru_delta": _ru_cache[key]})


def seconds_per_iteration(params, single_cta=False, team=0):
    """Measured seconds per CG iteration of the shape tune() chose."""
    tune(params, single_cta=single_cta, team=team)
    key = (params.L, params.Nt, round(params.beta / params.Nt, 12), single_cta, team, None)
    return _cache[key][1]


def simulate_batch(est_solo, est_team, is_team, num_ctas, csize):
    """Makespan of one batch step as the kernel schedules it: team chains
    first, by decreasing estimate, each taken by the next free cluster of
    csize CTAs; a cluster that finds no team chain left becomes csize
    independent CTAs; every CTA then takes the one-CTA chains in order of
    decreasing estimate as it becomes free."""
    import heapq
    nclus = num_ctas // csize if csize > 1 else 0
    teams = sorted((i for i in range(len(est_solo)) if is_team[i]), key=lambda i: -est_team[i])
    solos = sorted((i for i in range(len(est_solo)) if not is_team[i]), key=lambda i: -est_solo[i])
    if teams and nclus == 0:
        return float("inf")
    clus = [0.0] * nclus
    heapq.heapify(clus)
    end = 0.0
    for i in teams:
        t = heapq.heappop(clus) + est_team[i]
        end = max(end, t)
        heapq.heappush(clus, t)
    ctas = [t for t in clus for _ in range(csize)] if teams else []
    ctas += [0.0] * (num_ctas - len(ctas))
    heapq.heapify(ctas)
    for i in solos:
        t = heapq.heappop(ctas) + est_solo[i]
        end = max(end, t)
        heapq.heappush(ctas, t)
    return end


def plan_teams(est_solo, est_team, num_ctas, csize):
    """Which chains of a batch to run as cluster teams: the k most expensive
    (by one-CTA estimate), k chosen to minimise the simulated makespan.
    est_team[i] may be None for chains not worth a team.  Returns a list of
    booleans."""
    n = len(est_solo)
    cand = sorted((i for i in range(n) if est_team[i] is not None), key=lambda i: -est_solo[i])
    best_k, best = 0, simulate_batch(est_solo, est_team, [False] * n, num_ctas, csize)
    for k in range(1, len(cand) + 1):
        flags = [False] * n
        for i in cand[:k]:
            flags[i] = True
        m = simulate_batch(est_solo, est_team, flags, num_ctas, csize)
        if m < best:
            best_k, best = k, m
    flags = [False] * n
    for i in cand[:best_k]:
        flags[i] = True
    return flags


def batch_shapes(plist, csize=4, num_sms=None):
    """Launch shapes of a batch: each chain's tuned one-CTA shape, or a tuned
    cluster team of csize CTAs for the chains plan_teams picks, each with its
    tuned reliable-update threshold.  The time of a trajectory is estimated
    as the tuned seconds per CG iteration (one CTA, or the team) times Nt (at
    fixed delta the iterations per trajectory grow about in proportion to
    beta = Nt delta); teams are timed only for chains above half the ideal
    makespan."""
    if num_sms is None:
        dev = torch.device("cuda", torch.cuda.current_device())
        num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    solo = [tune(p, single_cta=True) for p in plist]
    est = [seconds_per_iteration(p, single_cta=True) * p.Nt for p in plist]
    ideal = sum(est) / max(1, num_sms)
    est_team = [seconds_per_iteration(p, team=csize) * p.Nt
                if csize > 1 and e > 0.5 * ideal else None for p, e in zip(plist, est)]
    teams = plan_teams(est, est_team, num_sms, csize) if csize > 1 else [False] * len(plist)
    shapes = [tune(p, team=csize) if t else s for p, s, t in zip(plist, solo, teams)]
    return [tune_ru(p) for p in shapes]
