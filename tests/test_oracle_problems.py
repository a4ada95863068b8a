"""The paper's problem set (Section 6.1) and its error measures, pinned on the CPU:
Helmholtz III's near-resonant reaction term against the spectrum of O1's assembled
matrix, the divergence-free field of Diffusion-Convection III, the two boundary vectors
of e1 / e2, and both errors of the oracle O2 against O1 on every problem (the paper's
Table error measures its method the same way against a full solve)."""
import numpy as np
import pytest

from oracle import nd_dense, o1
from paper_1302_5995_gb300 import inputs


def test_tenth_eigenvalue_is_the_assembled_matrix_spectrum():
    n = 12
    A = o1.assemble_dense(*inputs.laplace_fields(n), n)
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    for k in (1, 2, 3, 10, 57, n * n):
        assert abs(inputs.discrete_laplace_eigenvalue(n, k) - ev[k - 1]) < 1e-10 * ev[-1]


def test_helmholtz3_sits_1e_5_from_resonance():
    n = 12
    A = o1.assemble_dense(*inputs.paper_problem("helmholtz3", n), n)
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert abs(np.abs(ev).min() - 1e-5) < 1e-9


def test_problem_fields():
    n = 16
    X, Y = inputs.node_xy(n)
    b, c, _ = inputs.paper_problem("diffconv3", n)
    B, Cc = b.reshape(n, n), c.reshape(n, n)  # [j, i]
    assert np.ptp(B, axis=1).max() == 0.0 and np.ptp(Cc, axis=0).max() == 0.0  # b(y), c(x): divergence free
    b, c, _ = inputs.paper_problem("diffconv4", n)
    np.testing.assert_allclose(b, 125 * np.cos(4 * np.pi * X))
    np.testing.assert_allclose(c, 125 * np.sin(4 * np.pi * Y))
    _, _, d = inputs.paper_problem("helmholtz4", n)
    k = np.sqrt(-d[0])
    assert abs(2 * np.pi / (k / (n + 1)) - 40.0) < 1e-12  # 40 points per wavelength
    with pytest.raises(ValueError):
        inputs.paper_problem("nope", n)
    R = inputs.error_vectors(n, 3)
    np.testing.assert_allclose(np.linalg.norm(R, axis=0), 1.0)


def e12(V, V_ref):
    return np.linalg.norm(V - V_ref, axis=0) / np.linalg.norm(V_ref, axis=0)


@pytest.mark.parametrize("name", list(inputs.PAPER_PROBLEMS) + ["random1", "random2"])
def test_oracle_errors_on_the_problem_set(name):
    n, leaf = 20, 5
    R = inputs.error_vectors(n, 17)
    if name.startswith("random"):
        sx, sy = (inputs.random_laplacian_1 if name == "random1" else inputs.random_laplacian_2)(n)
        T, _ = nd_dense.build_loads(nd_dense.Problem.network(sx, sy, n), leaf, [])
        V_ref = o1.net_apply(sx, sy, n, R)
    else:
        b, c, d = inputs.paper_problem(name, n)
        T = nd_dense.build(b, c, d, n, leaf).T
        V_ref = o1.dtn_apply(b, c, d, n, R)
    e1, e2 = e12(T @ R, V_ref)
    bound = 1e-6 if name == "helmholtz3" else 1e-10  # condition ~ 1e8 near resonance
    assert e1 < bound and e2 < bound, (e1, e2)
