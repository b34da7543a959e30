"""Instance generator checks and the paper's dimension tables (CPU)."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

from oracle import opf
from paper_2301_04869_gb300 import synth

GOLD = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden", "paper_dimensions.txt")


def _rows(tag):
    out = []
    for line in open(GOLD):
        if line.startswith(tag + " "):
            out.append(line.split()[1:])
    return out


def test_table_instances_dimension_formulas():
    """n_x = 2 nbus - 1 - ngen and n_u = 2 ngen - 1 reproduce Table
    'MATPOWER instances' (Sec. 4.1.1) row by row."""
    rows = _rows("instances")
    assert len(rows) == 4
    for name, nb, nl, ng, nx, nu in rows:
        dx, du, m, _, _ = opf.dimensions(int(nb), int(nl), int(ng), 1, line_limits=True)
        assert (dx, du) == (int(nx), int(nu)), name


def test_table_dims_nvar_ncon():
    """nvar = N n_x + n_u, ncon = N (n_x + m) with line limits, and the
    K_uu size (Sec. 4.3 table).  The ncon of 1354pegase at N = 512 is printed
    as 4,425,280; the formula (and the N = 8 row scaled by 64) gives
    3,425,280, so that one entry is a typo in the table."""
    inst = {r[0]: r for r in _rows("instances")}
    for name, N, nvar, ncon, kmb in _rows("dims"):
        _, nb, nl, ng, _, _ = inst[name]
        nx, nu, m, dnvar, dncon = opf.dimensions(int(nb), int(nl), int(ng), int(N), line_limits=True)
        assert dnvar == int(nvar), name
        if name == "case1354pegase" and N == "512":
            assert dncon == 3425280 and int(ncon) - dncon == 1000000
        else:
            assert dncon == int(ncon), name
        assert abs(8.0 * nu * nu / 2**20 - float(kmb)) < 0.06, name


@pytest.mark.parametrize("n,ng", [(30, 6), (1000, 150)])
def test_network_shape(n, ng):
    net = synth.make_network(n, ng, seed=0)
    L = int(np.floor(1.35 * n + 0.5))
    assert net.n_line == L
    assert net.gen_bus[0] == 0 and len(set(net.gen_bus.tolist())) == ng
    A = sp.csr_matrix((np.ones(L), (net.fr, net.to)), shape=(n, n))
    assert connected_components(A, directed=False)[0] == 1
    keys = set(zip(np.minimum(net.fr, net.to).tolist(), np.maximum(net.fr, net.to).tolist()))
    assert len(keys) == L and np.all(net.fr != net.to)
    assert np.count_nonzero(net.pd0) <= int(np.floor(0.6 * n + 0.5))
    assert np.all((net.x / net.r >= 3) & (net.x / net.r <= 10))
    # deterministic
    net2 = synth.make_network(n, ng, seed=0)
    assert np.array_equal(net.fr, net2.fr) and np.array_equal(net.r, net2.r)


def test_scenarios_law():
    net = synth.make_network(200, 20, seed=0)
    pd, qd = synth.make_scenarios(net, 500, 0.05, seed=1)
    ratio = pd[:, net.load_bus] / net.pd0[net.load_bus]
    assert abs(ratio.mean() - 1.0) < 0.01 and abs(ratio.std() - 0.05) < 0.005
    assert np.all(pd >= 0)
    np.testing.assert_allclose(qd[:, net.load_bus] / pd[:, net.load_bus],
                               np.broadcast_to(net.qd0[net.load_bus] / net.pd0[net.load_bus], (500, net.load_bus.size)))
