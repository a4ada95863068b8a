"""The paper's problem set (Section 6.1: Laplace, Diffusion-Convection I-IV, Helmholtz
I-IV, Random Laplacian I-II) built on the GPU in FP64 through the C ABI, with the
paper's two error measures e1 (random unit boundary vector) and e2 (smooth one) against
O1's full solve.  Each tolerance is 100 times the spread between the oracle's own nested
dissection (O2) and O1 on the same problem, at least 1e-9: Helmholtz III sits 1e-5 from
resonance and Diffusion-Convection IV (a gradient convection field) is exponentially
ill-conditioned, so two exact methods already differ there."""
import numpy as np
import pytest

import paper_1302_5995_gb300 as gm
from oracle import nd_dense, o1
from paper_1302_5995_gb300 import inputs

pytestmark = pytest.mark.gpu

PROBLEMS = list(inputs.PAPER_PROBLEMS) + ["random1", "random2"]


def errors(V, V_ref):
    return np.linalg.norm(V - V_ref, axis=0) / np.linalg.norm(V_ref, axis=0)


@pytest.mark.parametrize("name", PROBLEMS)
@pytest.mark.parametrize("n,leaf", [(64, 8)])
def test_problem_set_e1_e2(name, n, leaf):
    R = inputs.error_vectors(n, 17)
    if name.startswith("random"):
        sx, sy = (inputs.random_laplacian_1 if name == "random1" else inputs.random_laplacian_2)(n)
        V_ref = o1.net_apply(sx, sy, n, R)
        T_o2, _ = nd_dense.build_loads(nd_dense.Problem.network(sx, sy, n), leaf, [])
        op = gm.build_network(sx, sy, n, leaf)
    else:
        b, c, d = inputs.paper_problem(name, n)
        V_ref = o1.dtn_apply(b, c, d, n, R)
        T_o2 = nd_dense.build(b, c, d, n, leaf).T
        op = gm.build(b, c, d, n, leaf)
    spread = errors(T_o2 @ R, V_ref).max()
    V = op.solve(np.ascontiguousarray(R.T)).T
    e1, e2 = errors(V, V_ref)
    bound = max(1e-9, 100.0 * spread)
    assert e1 < bound and e2 < bound, (name, e1, e2, spread)


@pytest.mark.parametrize("name", ["laplace", "diffconv1", "diffconv3", "helmholtz1", "random1", "random2"])
def test_hbs_memory_per_n_stays_flat(name):
    """The paper's compressibility claim (Table mem): the memory M(n) of the solution
    operator in HBS form grows like n, so M(n)/n stays about flat from n = 256 to 1024
    (within 1.6x; 2.5x for the convection problems, twice as convection-dominated here
    as in the textbook scheme under the literal 1/h reading, whose boundary layers add
    rank as the grid resolves them)."""
    ratios = []
    for n in (256, 512, 1024):
        try:
            if name.startswith("random"):
                sx, sy = (inputs.random_laplacian_1 if name == "random1" else inputs.random_laplacian_2)(n)
                inf = gm.build_network(sx, sy, n, 16, tol=1e-7, hbs_leaf=64).info()
            else:
                b, c, d = inputs.paper_problem(name, n)
                inf = gm.build(b, c, d, n, 16, tol=1e-7, hbs_leaf=64).info()
        except gm.GmError as e:  # a node rank at the documented cap of the GPU sampling
            if (name.startswith("diffconv") or name == "random2") and e.code == gm.GM_EUNSUPPORTED:
                pytest.skip(f"{name}: an HBS rank reached the cap at n = {n}")
            raise
        if name.startswith("diffconv") and inf["hbs_fallbacks"] > 0 and inf["hbs_levels"] == 0:
            # Algorithm 1's inverse of this convection-dominated root failed its residual
            # check and the root was eliminated densely: there is no HBS operator to weigh
            pytest.skip(f"{name}: the HBS root inverse was refused (unstable) at n = {n}")
        assert inf["hbs_levels"] > 0 and 0 < inf["hbs_operator_bytes"] <= inf["hbs_bytes"]
        ratios.append(inf["hbs_operator_bytes"] / n)
    assert ratios[2] < (2.5 if name.startswith("diffconv") else 1.6) * ratios[0], ratios


def test_server_serves_an_hbs_operator():
    """A served operator in HBS form answers through Algorithm 2 what the dense operator
    of the same problem answers (within the compression tolerance)."""
    n = 256
    b, c, d = inputs.paper_problem("laplace", n)
    dense = gm.build(b, c, d, n, 16)
    srv = gm.Server(1 << 36)
    oid = srv.add(gm.build(b, c, d, n, 16, tol=1e-9, hbs_leaf=64))
    G = np.ascontiguousarray(inputs.gaussian_vectors(n, 8, 21).T)  # vector j contiguous
    out = np.zeros_like(G)
    assert srv.wait(srv.submit(oid, G, out, 8)) == 0
    ref = dense.solve(G)
    assert np.abs(out - ref).max() / np.abs(ref).max() < 1e-7
    st = srv.stats()
    assert st["requests"] == 1 and st["vectors"] == 8 and st["resident_bytes"] > 0
    srv.close()


@pytest.mark.parametrize("make", [inputs.random_laplacian_1, inputs.random_laplacian_2])
def test_network_with_hbs_root_matches_the_dense_network(make):
    """A network's root in HBS form (the datum rows weighted by the ghosts' conductivities
    in every apply) against the dense network build, within 100 tol."""
    n, leaf, tol = 128, 16, 1e-9
    sx, sy = make(n)
    T = gm.build_network(sx, sy, n, leaf).dtn()
    try:
        op = gm.build_network(sx, sy, n, leaf, tol=tol, hbs_leaf=32)
    except gm.GmError as e:  # the 1:1000 contrast may lift a node rank to the sampling cap
        if make is inputs.random_laplacian_2 and e.code == gm.GM_EUNSUPPORTED:
            pytest.skip("Random Laplacian II: an HBS rank reached the cap")
        raise
    assert op.info()["hbs_levels"] > 0
    assert np.abs(op.dtn() - T).max() / np.abs(T).max() < 100 * tol
    G = np.ascontiguousarray(inputs.gaussian_vectors(n, 4, 23).T)
    assert np.abs(op.solve(G) - (T @ G.T).T).max() / np.abs(T @ G.T).max() < 100 * tol


def test_server_builds_an_operator_and_serves_solves_queued_behind_it():
    """A build request on the server's worker, a solve submitted for the new operator
    before the build finished, and the result equal to a direct build's solve."""
    n, leaf = 64, 8
    b, c, d = inputs.convection_fields(n, seeds=(3, 4, 5))
    ref = gm.build(b, c, d, n, leaf)
    srv = gm.Server(1 << 34)
    oid, rb = srv.submit_build(b, c, d, n, leaf)
    G = np.ascontiguousarray(inputs.gaussian_vectors(n, 4, 31).T)  # vector j contiguous
    out = np.zeros_like(G)
    rs = srv.submit(oid, G, out, 4)
    assert srv.wait(rs) == 0 and srv.wait(rb) == 0
    assert srv.poll(rb) == (True, 0)
    V = ref.solve(G)
    assert np.abs(out - V).max() <= 1e-12 * np.abs(V).max()
    assert srv.stats()["resident_ops"] == 1
    srv.close()
