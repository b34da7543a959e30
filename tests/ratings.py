"""Line ratings for the tests of the line-flow limits of §4.1.1.

The synthetic networks carry no ratings of their own (the paper's MATPOWER
cases do).  Here they come from the unconstrained optimum found by the
oracle: every line is rated at 1.2 times the larger of its two end flows
(at least 0.05 pu), and the `tight` most loaded lines at 0.9 times it, so
those limits bind at the new optimum."""
import numpy as np

from oracle import ipm as oipm
from oracle import opf
from paper_2301_04869_gb300 import synth

_cache = {}


def end_flows(M, x, u):
    """max(|S_f|, |S_t|) per line at (x, u) of scenario 0."""
    th, v = opf.bus_voltage(M.lay, x, u)
    Yf, Yt, Cf, Ct = opf.branch_admittance(M.net)
    return np.maximum(np.abs(opf.branch_flows(Yf, Cf, th, v)), np.abs(opf.branch_flows(Yt, Ct, th, v)))


def rated(n, ng, N, sigma, tight=3):
    """(net with ratings, pd, qd) for a network of n buses; N scenarios."""
    key = (n, ng, N, sigma, tight)
    if key not in _cache:
        net = synth.make_network(n, ng, seed=0)
        pd, qd = synth.make_scenarios(net, N, sigma, seed=1)
        M = opf.Model(net, pd[:1], qd[:1])
        st, _, _ = oipm.solve(M)
        flows = end_flows(M, st["x"][0], st["u"])
        _cache[key] = (synth.with_ratings(net, flows, tight=tight), pd, qd)
    return _cache[key]
