"""Host logic of the autotuner (no GPU): candidate shapes and the choice."""
from paper_2210_06874_gb300 import autotune, hmc


def test_candidates_cover_one_cta_and_tile_teams():
    p = hmc.Params(L=6, Nt=32, beta=4.0)
    c = autotune.candidates(p, num_sms=148)
    assert (1, 1, 32) in c and (12, 1, 8) in c and (12, 4, 8) in c
    assert all(ns in (8, 16, 32) for _, _, ns in c)
    assert all(inner <= team <= 148 for team, inner, _ in c)
    single = autotune.candidates(p, num_sms=148, single_cta=True)
    assert single == [(1, 1, 8), (1, 1, 16), (1, 1, 32)]


def test_pick_fastest_then_fewest_ctas():
    t = [((12, 4, 8), 2.0e-5), ((12, 1, 32), 2.3e-5), ((4, 4, 8), 2.0e-5)]
    assert autotune.pick(t) == (4, 4, 8)
