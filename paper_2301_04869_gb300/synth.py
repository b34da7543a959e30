"""Seeded synthetic power networks and load scenarios.

This module only draws data: bus/line/generator parameters and per-scenario
loads.  It holds none of the interior-point arithmetic, so both the CUDA path
and the CPU oracle can be fed from it without sharing any of the method.

The paper benchmarks MATPOWER cases (Table "MATPOWER instances", §4.1.1),
which are not available here; the networks below stand in for them with the
same structure: a connected meshed grid (mean degree 2.7), generators on a
subset of buses with the slack generator at bus 0, loads on 60 % of the buses,
and N load scenarios sharing one network (§4.1.1: each scenario is assigned its
own load parameters).

Draw order (fixed, one ``numpy.random.default_rng`` stream per seed):
tree -> chords -> line parameters -> load buses -> P -> Q factors ->
generator buses -> generator parameters.  Scenario factors come from a second
stream (scenario seed).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Network:
    """One synthetic network in per-unit.  Lines use the pi model with no taps.

    Arrays (all numpy):
      fr, to      int32[L]   line end buses (fr = parent for tree lines)
      r, x, b     float64[L] series resistance, reactance, total charging
      gen_bus     int32[n_g] bus of each generator; gen_bus[0] == 0 (slack)
      pmax        float64[n_g] (pmin = 0)
      qmax        float64[n_g] (qmin = -qmax)
      c2, c1      float64[n_g] quadratic cost coefficients
      vmin, vmax  float64[n]
      pd0, qd0    float64[n] base loads
      rate        float64[L] apparent-power rating of every line, or None
                  (no line-flow limits; see ``with_ratings``)
    """
    n_bus: int
    fr: np.ndarray
    to: np.ndarray
    r: np.ndarray
    x: np.ndarray
    b: np.ndarray
    gen_bus: np.ndarray
    pmax: np.ndarray
    qmax: np.ndarray
    c2: np.ndarray
    c1: np.ndarray
    vmin: np.ndarray
    vmax: np.ndarray
    pd0: np.ndarray
    qd0: np.ndarray
    load_bus: np.ndarray
    seed: int = 0
    rate: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n_line(self) -> int:
        return int(self.fr.shape[0])

    @property
    def n_gen(self) -> int:
        return int(self.gen_bus.shape[0])


LOAD_SCALE = 0.3


def _round_half_up(v: float) -> int:
    return int(math.floor(v + 0.5))


def make_network(n_bus: int, n_gen: int | None = None, seed: int = 0,
                 line_ratio: float = 1.35, load_frac: float = 0.6,
                 load_scale: float = LOAD_SCALE) -> Network:
    """Draw one network: a random spanning tree plus uniform chords.

    The spanning tree is a random recursive tree (bus k attaches to a uniform
    earlier bus); the L - (n-1) chords are uniform over bus pairs that are not
    yet adjacent, without repeats, so that L = floor(1.35 n + 1/2) (mean
    degree 2.7).  Loads sit on floor(0.6 n + 1/2) distinct buses with
    P ~ load_scale * U(0,1), Q = P * U(0.2, 0.4).  With the stated line laws
    (x ~ 0.16 pu on average, R/X up to 1/3) an unscaled load density is past
    the power-flow solvability limit of these grids, so every workload uses
    load_scale = 0.3 (one constant for all sizes).
    Generators: slack at bus 0 plus n_g - 1 distinct non-slack buses, with
    Pg in [0, U(1,5)], Qg in +-U(0.5, 2), costs c2 ~ U(0.001, 0.1),
    c1 ~ U(1, 40); V in [0.9, 1.1] at every bus.
    """
    n = int(n_bus)
    if n < 2:
        raise ValueError("need at least two buses")
    if n_gen is None:
        n_gen = max(1, _round_half_up(0.1 * n))
    n_gen = int(n_gen)
    if not 1 <= n_gen <= n:
        raise ValueError("bad generator count")
    L = _round_half_up(line_ratio * n)
    if L < n - 1 or L > n * (n - 1) // 2:
        raise ValueError("bad line count")
    rng = np.random.default_rng(seed)

    # tree: bus k attaches to a uniform earlier bus (random recursive tree)
    parents = rng.integers(0, np.arange(1, n))
    fr = list(parents.tolist())
    to = list(range(1, n))
    adj = set()
    for a_, c_ in zip(fr, to):
        adj.add((min(a_, c_), max(a_, c_)))
    # chords: uniform over bus pairs not yet adjacent, without repeats
    need = L - (n - 1)
    while need > 0:
        pairs = rng.integers(0, n, size=(max(2 * need, 16), 2))
        for a_, c_ in pairs.tolist():
            if need == 0:
                break
            if a_ == c_:
                continue
            key = (min(a_, c_), max(a_, c_))
            if key in adj:
                continue
            adj.add(key)
            fr.append(a_)
            to.append(c_)
            need -= 1
    fr = np.asarray(fr, dtype=np.int32)
    to = np.asarray(to, dtype=np.int32)

    r = rng.uniform(0.001, 0.05, L)
    x = r * rng.uniform(3.0, 10.0, L)
    b = rng.uniform(0.0, 0.05, L)

    n_load = _round_half_up(load_frac * n)
    load_bus = np.sort(rng.choice(n, size=n_load, replace=False)).astype(np.int32)
    p_load = load_scale * rng.uniform(0.0, 1.0, n_load)
    q_fac = rng.uniform(0.2, 0.4, n_load)
    pd0 = np.zeros(n)
    qd0 = np.zeros(n)
    pd0[load_bus] = p_load
    qd0[load_bus] = p_load * q_fac

    others = rng.choice(np.arange(1, n), size=n_gen - 1, replace=False)
    gen_bus = np.concatenate([[0], np.sort(others)]).astype(np.int32)
    pmax = rng.uniform(1.0, 5.0, n_gen)
    qmax = rng.uniform(0.5, 2.0, n_gen)
    c2 = rng.uniform(0.001, 0.1, n_gen)
    c1 = rng.uniform(1.0, 40.0, n_gen)

    return Network(n_bus=n, fr=fr, to=to, r=r, x=x, b=b, gen_bus=gen_bus,
                   pmax=pmax, qmax=qmax, c2=c2, c1=c1,
                   vmin=np.full(n, 0.9), vmax=np.full(n, 1.1),
                   pd0=pd0, qd0=qd0, load_bus=load_bus, seed=seed)


def with_ratings(net: Network, flows: np.ndarray, factor: float = 1.2, floor: float = 0.05,
                 tight: int = 0, tight_factor: float = 0.9) -> Network:
    """A copy of ``net`` with line ratings (the operational limits of §4.1.1,
    |S| <= rate at both ends of every line).  The paper's MATPOWER cases carry
    their own ratings; here they are drawn from a reference flow: ``flows``
    (float64[L], e.g. the larger end's apparent power at an unconstrained
    optimum) times ``factor``, at least ``floor`` pu, and the ``tight`` most
    loaded lines get ``tight_factor`` times their flow instead, so that those
    limits bind.  Only the ratings are new; every other array is shared."""
    import copy
    flows = np.asarray(flows, dtype=np.float64)
    rate = np.maximum(factor * flows, floor)
    if tight > 0:
        top = np.argsort(-flows, kind="stable")[:tight]
        rate[top] = np.maximum(tight_factor * flows[top], floor)
    out = copy.copy(net)
    out.rate = rate
    out.meta = dict(net.meta)
    return out


def bridges(net: Network) -> np.ndarray:
    """Boolean mask of the lines whose loss disconnects the network (graph
    bridges, by depth-first search low-link values)."""
    n, L = net.n_bus, net.n_line
    adj = [[] for _ in range(n)]
    for l in range(L):
        a, b = int(net.fr[l]), int(net.to[l])
        adj[a].append((b, l))
        adj[b].append((a, l))
    disc = [-1] * n
    low = [0] * n
    out = np.zeros(L, dtype=bool)
    t = 0
    for root in range(n):
        if disc[root] >= 0:
            continue
        disc[root] = low[root] = t
        t += 1
        stack = [(root, -1, iter(adj[root]))]
        while stack:
            v, pl, it = stack[-1]
            nxt = next(it, None)
            if nxt is None:
                stack.pop()
                if stack:
                    p = stack[-1][0]
                    low[p] = min(low[p], low[v])
                    if low[v] > disc[p]:
                        out[pl] = True
                continue
            w, l = nxt
            if l == pl:
                continue
            if disc[w] < 0:
                disc[w] = low[w] = t
                t += 1
                stack.append((w, l, iter(adj[w])))
            else:
                low[v] = min(low[v], disc[w])
    return out


def make_contingencies(net: Network, n_scen: int, frac: float = 0.5, seed: int = 2) -> np.ndarray:
    """Line-tripping contingencies (§4.1.1: a scenario carries its loads and
    potential line trips): scenario 0 keeps the intact network; each other
    scenario, with probability ``frac``, loses one line drawn uniformly from
    the lines whose loss keeps the network connected.  Returns int32[n_scen],
    the tripped line or -1."""
    rng = np.random.default_rng(seed)
    cand = np.flatnonzero(~bridges(net))
    trip = np.full(int(n_scen), -1, dtype=np.int32)
    if cand.size == 0:
        return trip
    pick = rng.uniform(size=int(n_scen)) < frac
    lines = rng.choice(cand, size=int(n_scen))
    trip[pick] = lines[pick]
    trip[0] = -1
    return trip


def make_scenarios(net: Network, n_scen: int, sigma: float, seed: int = 1):
    """Per-scenario loads: each loaded bus gets its own factor 1 + sigma*N(0,1),
    clipped at 0, applied to both P and Q.  sigma = 0 returns the base loads.
    Returns (pd, qd), each float64[n_scen, n_bus], scenario-major."""
    n_scen = int(n_scen)
    rng = np.random.default_rng(seed)
    nl = net.load_bus.shape[0]
    if sigma > 0:
        fac = 1.0 + sigma * rng.standard_normal((n_scen, nl))
        fac = np.maximum(fac, 0.0)
    else:
        fac = np.ones((n_scen, nl))
    pd = np.zeros((n_scen, net.n_bus))
    qd = np.zeros((n_scen, net.n_bus))
    pd[:, net.load_bus] = fac * net.pd0[net.load_bus][None, :]
    qd[:, net.load_bus] = fac * net.qd0[net.load_bus][None, :]
    return pd, qd


def capacity_margin(net: Network, pd: np.ndarray) -> float:
    """(sum Pmax) / max over scenarios of (sum Pd) - 1."""
    tot = pd.sum(axis=1).max()
    return float(net.pmax.sum() / max(tot, 1e-300) - 1.0)


def screened_network(n_bus, n_gen, n_scen, sigma, seed=0, scen_seed=1,
                     min_margin=0.03, max_tries=100000, load_scale=LOAD_SCALE):
    """Draw networks at seed, seed+1, ... until total generator capacity
    exceeds the largest scenario's total load by ``min_margin`` (the stated
    laws give capacity ~= load at 10 % generator buses, so some draws cannot
    be feasible).  Returns (net, pd, qd); ``net.seed`` records the seed used."""
    for t in range(max_tries):
        net = make_network(n_bus, n_gen, seed=seed + t, load_scale=load_scale)
        pd, qd = make_scenarios(net, n_scen, sigma, seed=scen_seed)
        if capacity_margin(net, pd) >= min_margin:
            net.meta["seed_tries"] = t + 1
            return net, pd, qd
    raise RuntimeError("no network passed the capacity screen")


# Workloads (sizes of the paper's instance class, Table "MATPOWER instances").
# Load scale per workload: the 30-bus network solves with the stated load law
# (scale 1); the 1000-bus network does not (the interior-point method's primal
# residual stalls at 1.5 pu while its multipliers diverge) and takes 0.3; the
# 10,000-bus network (generators at 10 % of its buses, against 15 % on the
# 1000-bus one) is still past solvability at 0.3 (every draw tried, seeds
# 0-6, stalls the same way) and takes 0.2.
CONFIGS = {
    # name: (n_bus, n_gen, n_scen, sigma, min_margin, load_scale)
    "opf30_n1": (30, 6, 1, 0.0, 0.03, 1.0),
    "opf1000_n64": (1000, 150, 64, 0.05, 0.03, LOAD_SCALE),
    "opf10000_n256": (10000, 1000, 256, 0.05, 0.03, 0.2),
}


def workload(name: str, n_scen: int | None = None):
    """Return (net, pd, qd) for a named workload; ``n_scen`` optionally takes
    the first scenarios of the workload's scenario draw."""
    n_bus, n_gen, N, sigma, margin, scale = CONFIGS[name]
    net, pd, qd = screened_network(n_bus, n_gen, N, sigma, seed=0, scen_seed=1,
                                   min_margin=margin, load_scale=scale)
    if n_scen is not None:
        pd = pd[:n_scen].copy()
        qd = qd[:n_scen].copy()
    return net, pd, qd


def uneven_batch(n_inst=512, seed=4, nmin=100, nmax=5000, smin=8, smax=128,
                 min_margin=0.03):
    """Many independent networks: bus counts log-uniform in [nmin, nmax],
    generators at 10 % of buses, scenario counts uniform in {smin..smax}.
    Returns a list of (net, pd, qd)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(nmin), math.log(nmax), n_inst))
    sizes = np.array([_round_half_up(s) for s in sizes])
    scen = rng.integers(smin, smax + 1, n_inst)
    out = []
    for j in range(n_inst):
        n = int(sizes[j])
        ng = max(2, _round_half_up(0.1 * n))
        out.append(screened_network(n, ng, int(scen[j]), 0.05,
                                    seed=100000 * (j + 1), scen_seed=1 + j,
                                    min_margin=min_margin))
    return out
