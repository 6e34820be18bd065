"""Pins for the oracle's deterministic label propagation (Sec. 11,
"Deterministic Label Propagation Refinement", with the gain of Sec. 6).

Pins: the move-conflict example of Sec. 6 (weights 5 and 2 from the figure
caption) worked by hand; candidate moves against the exhaustively pinned
gains; single-move gain exactness; applied sets as (gain desc, id asc)
prefixes; the chosen state against a merge path built independently with
Python's stable sort, and its maximality; balance; the all-feasible special
case; incremental pin counts against a rebuild.
"""
import json
import os

import numpy as np
import pytest

import synth
from tests.tiny import from_nets, random_hypergraph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_move_conflict_example(oracle_mod):
    g = load_golden("move_conflict.json")
    hg = from_nets(g["n"], g["nets"], g["net_w"], g["node_w"])
    k = g["k"]
    part = np.array(g["part"], np.int32)
    assert oracle_mod.objective(hg, k, part) == g["objective_before"]
    new_part, mv = oracle_mod.lp_subround(hg, k, part, g["eps_ppm"], 1, 1, 0, 0, 0)
    got = {int(u): (int(t), int(x)) for u, t, x in zip(mv["u"], mv["dst"], mv["gain"])}
    assert got == {int(u): tuple(v) for u, v in g["candidates"].items()}
    assert sorted(mv["u"][mv["applied"]].tolist()) == g["applied"]
    assert oracle_mod.objective(hg, k, new_part) == g["objective_after"]
    # second sub-round from the new state (hand-worked as well)
    part2, mv2 = oracle_mod.lp_subround(hg, k, new_part, g["eps_ppm"], 1, 1, 0, 1, 0)
    got2 = {int(u): (int(t), int(x)) for u, t, x in zip(mv2["u"], mv2["dst"], mv2["gain"])}
    assert got2 == {int(u): tuple(v) for u, v in g["second"]["candidates"].items()}
    assert sorted(mv2["u"][mv2["applied"]].tolist()) == g["second"]["applied"]
    assert oracle_mod.objective(hg, k, part2) == g["second"]["objective_after"]


def merge_path(A, B):
    """States (i, j) visited when merging the non-decreasing sequences
    A[0..a-1] and B[0..b-1], ties taken from A (built with a stable sort)."""
    items = [(A[i], 0, i) for i in range(len(A) - 1)] + [(B[j], 1, j) for j in range(len(B) - 1)]
    items.sort(key=lambda x: (x[0], x[1]))
    states = [(0, 0)]
    i = j = 0
    for _, which, _ in items:
        if which == 0:
            i += 1
        else:
            j += 1
        states.append((i, j))
    return states


def check_subround(oracle_mod, hg, k, part, eps_ppm, S, seed, level, pass_, s):
    W = int(hg.node_w.sum())
    lmax = oracle_mod.balance_limit(W, k, eps_ppm)
    bw = oracle_mod.block_weights(hg, k, part)
    new_part, mv = oracle_mod.lp_subround(hg, k, part, eps_ppm, S, seed, level, pass_, s)
    gains = oracle_mod.gains(hg, k, part)
    c = hg.node_w.astype(np.int64)
    # candidates: every node of the sub-round with a positive best gain, best
    # target by (gain desc, block asc)
    in_sr = [u for u in range(hg.n) if oracle_mod.subround_lp(seed, level, pass_, u, S) == s]
    cand = {int(u): (int(t), int(g)) for u, t, g in zip(mv["u"], mv["dst"], mv["gain"])}
    for u in in_sr:
        row = gains[u].copy()
        row[part[u]] = np.iinfo(np.int64).min
        best = int(row.max())
        if best > 0:
            assert cand[u] == (int(np.flatnonzero(row == best)[0]), best)
        else:
            assert u not in cand
    assert set(cand) <= set(in_sr)
    applied = {int(u) for u in mv["u"][mv["applied"]]}
    # per block pair: prefixes in (gain desc, id asc) order, last feasible state on the path
    for a in range(k):
        for b in range(a + 1, k):
            Mab = sorted([u for u in cand if part[u] == a and cand[u][0] == b],
                         key=lambda u: (-cand[u][1], u))
            Mba = sorted([u for u in cand if part[u] == b and cand[u][0] == a],
                         key=lambda u: (-cand[u][1], u))
            ia = sum(u in applied for u in Mab)
            jb = sum(u in applied for u in Mba)
            assert all(u in applied for u in Mab[:ia]) and all(u in applied for u in Mba[:jb])
            A = np.concatenate([[0], np.cumsum(c[Mab])]) if Mab else np.array([0])
            B = np.concatenate([[0], np.cumsum(c[Mba])]) if Mba else np.array([0])
            sa = max(0, lmax - int(bw[a])) // (k - 1)
            sb = max(0, lmax - int(bw[b])) // (k - 1)
            feas = [st for st in merge_path(A, B) if -sa <= A[st[0]] - B[st[1]] <= sb]
            assert feas[-1] == (ia, jb)
    # moves applied as chosen, nothing else changed
    for u in range(hg.n):
        if u in applied:
            assert new_part[u] == cand[u][0]
        else:
            assert new_part[u] == part[u]
    # balance holds after the sub-round when it held before
    if np.all(bw <= lmax):
        assert np.all(oracle_mod.block_weights(hg, k, new_part) <= lmax)
    # a lone applied move changes the objective by exactly its gain
    if len(applied) == 1:
        (u,) = applied
        f0 = oracle_mod.objective(hg, k, part)
        f1 = oracle_mod.objective(hg, k, new_part)
        assert f0 - f1 == cand[u][1]
    return new_part, len(applied), len(cand)


@pytest.mark.parametrize("k,seed", [(2, 1), (3, 2), (4, 3), (8, 4)])
def test_subround_rules_random(oracle_mod, k, seed):
    rng = np.random.default_rng(seed)
    hg = random_hypergraph(rng, 120, 160, 6, w_hi=6, c_hi=4)
    part = oracle_mod.initial_partition(hg.node_w, k, seed)
    S = 3
    total_applied = 0
    for pass_ in range(2):
        for s in range(S):
            part, na, nc = check_subround(oracle_mod, hg, k, part, 30000, S, seed, 0, pass_, s)
            total_applied += na
    assert total_applied > 0


def test_single_move_subrounds(oracle_mod):
    # with many sub-rounds most sub-rounds apply at most one move; each lone
    # move is checked against the objective difference inside check_subround
    hg = synth.random_uniform(3, 150, 200, node_w=(1, 3), net_w=(1, 5))
    k = 3
    part = oracle_mod.initial_partition(hg.node_w, k, 3)
    lone = 0
    S = 40
    for pass_ in range(3):
        for s in range(S):
            part, na, _ = check_subround(oracle_mod, hg, k, part, 30000, S, 3, 0, pass_, s)
            lone += na == 1
    assert lone >= 3


def test_all_moves_feasible_with_large_slack(oracle_mod):
    # eps = 100 %: L_max = 2 ceil(W/k) >= W, so every state on every merge path
    # is feasible (k = 2) and all candidate moves are applied
    hg = synth.random_uniform(8, 300, 300)
    part = oracle_mod.initial_partition(hg.node_w, 2, 8)
    _, mv = oracle_mod.lp_subround(hg, 2, part, 1_000_000, 4, 8, 0, 0, 1)
    assert len(mv["u"]) > 0 and mv["applied"].all()


@pytest.mark.parametrize("k", [2, 8])
def test_refine_incremental_state(oracle_mod, k):
    hg = synth.random_uniform(12, 2000, 2000, node_w=(1, 4), net_w=(1, 9))
    part0 = oracle_mod.initial_partition(hg.node_w, k, 12)
    res = oracle_mod.lp_refine(hg, k, part0, 30000, 8, 12, 0, 5, want_phi=True, want_trace=True)
    phi, _ = oracle_mod.pin_counts(hg, k, res["part"])
    assert np.array_equal(res["phi"], phi)
    assert res["objective"] == oracle_mod.objective(hg, k, res["part"])
    assert res["objective"] < oracle_mod.objective(hg, k, part0)
    lmax = oracle_mod.balance_limit(int(hg.node_w.sum()), k, 30000)
    assert np.all(oracle_mod.block_weights(hg, k, res["part"]) <= lmax)
    assert res["moves"] == int(res["applied"].sum())
    # early stop: passes run until one applies nothing
    applied_per_pass = res["applied"].sum(axis=1)
    assert res["passes"] == 5 or applied_per_pass[res["passes"] - 1] == 0
    # determinism
    again = oracle_mod.lp_refine(hg, k, part0, 30000, 8, 12, 0, 5)
    assert np.array_equal(again["part"], res["part"])
