"""Host logic of the autotuner (no GPU): candidate shapes and the choice."""
from paper_2210_06874_gb300 import autotune, hmc


def test_candidates_cover_one_cta_and_tile_teams():
    p = hmc.Params(L=6, Nt=32, beta=4.0)
    c = autotune.candidates(p, num_sms=148)
    assert (1, 1, 32, 1) in c and (12, 1, 8, 1) in c and (12, 4, 8, 1) in c
    assert (12, 1, 16, 2) in c                   # resident E, one site block
    assert all(ns in (8, 16, 32) for _, _, ns, m in c if m != 4)
    assert (12, 1, 0, 4) in c and (12, 8, 0, 4) in c   # slice-major, slices chosen by the library
    assert all(inner <= team <= 148 for team, inner, _, m in c if m != 5)
    assert not any(m == 5 for *_, m in c)            # split-K tiles: V >= 128 only
    single = autotune.candidates(p, num_sms=148, single_cta=True)
    assert single == [(1, 1, 0, 4), (1, 1, 8, 1), (1, 1, 8, 2), (1, 1, 16, 1), (1, 1, 16, 2),
                      (1, 1, 32, 1)]
    big = autotune.candidates(hmc.Params(L=24, Nt=96, beta=12.0), num_sms=148)
    assert all(mode in (1, 4, 5) for *_, mode in big)  # E rows too large to stay resident
    # split-K tiles: clusters of 2..8 CTAs, n-groups of the library's size or
    # of 32 or 16 slices, the launch size left to the library
    assert sorted(s for s in big if s[3] == 5) == sorted(
        (0, C, ns, 5) for C in (2, 4, 6, 8) for ns in (0, 16, 32))
    small_nt = autotune.candidates(hmc.Params(L=12, Nt=16, beta=2.0), num_sms=148)
    assert sorted(s for s in small_nt if s[3] == 5) == sorted(
        (0, C, 0, 5) for C in (2, 4, 6, 8))            # n-groups smaller than Nt only
    assert (0, 6, 0, 5) not in autotune.candidates(hmc.Params(L=6, Nt=32, beta=4.0),
                                                   num_sms=148, single_cta=True)


def test_pick_fastest_then_fewest_ctas():
    t = [((12, 4, 8, 1), 2.0e-5), ((12, 1, 32, 2), 2.3e-5), ((4, 4, 8, 1), 2.0e-5)]
    assert autotune.pick(t) == (4, 4, 8, 1)


def test_small_cluster_mode_candidates():
    """CUDA-core cluster mode (operand_mode 3): clusters of 1, 2, 4, 8 CTAs with
    at most 16 slices each and the layout inside the 208 KB operand area."""
    c = autotune.candidates(hmc.Params(L=6, Nt=32, beta=4.0), num_sms=148)
    small = [s for s in c if s[3] == 3]
    assert (8, 8, 8, 3) in small and (2, 2, 8, 3) in small
    assert all(team % inner == 0 for team, inner, _, _ in small)
    assert not any(inner == 1 for _, inner, _, _ in small)     # 32 slices on one CTA
    assert autotune.small_feasible(72, 32, 8)
    assert not autotune.small_feasible(72, 32, 1)
    assert autotune.small_feasible(128, 64, 8)                   # L = 8
    assert not autotune.small_feasible(1152, 96, 8)              # L = 24: E^T too large
    assert not autotune.small_feasible(18, 4, 8)                 # fewer slices than CTAs
    big = autotune.candidates(hmc.Params(L=24, Nt=96, beta=12.0), num_sms=148)
    assert not any(mode == 3 for *_, mode in big)


def test_team_candidates_and_plan():
    """Cluster-team shapes keep every CTA in the inner team; the chains whose
    one-CTA estimate exceeds the batch's ideal makespan become teams."""
    p = hmc.Params(L=12, Nt=64, beta=8.0)
    c = autotune.team_candidates(p, 4)
    assert (4, 4, 0, 4) in c and (4, 4, 8, 1) in c
    assert all(team == inner == 4 for team, inner, _, _ in c)
    assert not any(m == 3 for *_, m in c)                          # V = 288: no CUDA-core mode
    assert (4, 4, 8, 3) in autotune.team_candidates(hmc.Params(L=6, Nt=32, beta=4.0), 4)
    # one long chain: as a team of 4 (3.0) it no longer sets the makespan
    est = [10.0] + [1.0] * 8
    team = [3.0] + [None] * 8
    assert autotune.plan_teams(est, team, 8, 4) == [True] + [False] * 8
    assert autotune.simulate_batch(est, team, [True] + [False] * 8, 8, 4) == 3.0
    assert autotune.simulate_batch(est, team, [False] * 9, 8, 4) == 10.0
    assert autotune.plan_teams([1.0] * 8, [0.4] * 8, 8, 4) == [False] * 8   # balanced: none
    # more team chains than clusters pay a second wave: 6 teams on 4 clusters
    # end at 6.0, the best choice here; the planner takes the k with the
    # smallest simulated makespan
    est = [8.0] * 6 + [1.0] * 8
    team = [3.0] * 6 + [None] * 8
    flags = autotune.plan_teams(est, team, 16, 4)
    m = autotune.simulate_batch(est, team, flags, 16, 4)
    assert m == min(autotune.simulate_batch(est, team, [i < k for i in range(14)], 16, 4)
                    for k in range(7)) == 6.0
    # a slow team (6.0 of 8.0) does not pay for its second wave
    assert autotune.plan_teams([8.0] * 6, [6.0] * 6, 16, 4) == [False] * 6
