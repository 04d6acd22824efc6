"""Pins of the Kron-reduction oracle (Sec. IV-A, compressed Laplacians as
the Schur complement onto the sampled nodes) against facts that do not
reuse its LU solve: closed forms of electrical networks, effective
resistances, a least-squares energy minimisation, the quotient property,
the connectivity theorem the paper cites, and Laplacian invariants."""
from collections import deque

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import oracle as O
from oracle import cpca_kron as KR


def _random_graph(N, rng, deg=3):
    """Connected symmetric weights: a path through a random permutation plus
    random chords, weights in [0.2, 1]."""
    W = np.zeros((N, N))
    perm = rng.permutation(N)
    for a, b in zip(perm[:-1], perm[1:]):
        W[a, b] = W[b, a] = rng.uniform(0.2, 1.0)
    for _ in range(deg * N // 2):
        i, j = rng.choice(N, 2, replace=False)
        W[i, j] = W[j, i] = rng.uniform(0.2, 1.0)
    return W


def _lap(W, lap_type=O.LAP_COMBINATORIAL):
    return O.laplacian_from_weights(sp.csr_matrix(W), lap_type)


def test_path_series_closed_form():
    """Eliminating the interior nodes of a path leaves resistors in series:
    conductance 1 / (1/w1 + 1/w2)."""
    w = [0.5, 2.0, 0.25, 4.0]
    W = np.zeros((5, 5))
    for i, wi in enumerate(w):
        W[i, i + 1] = W[i + 1, i] = wi
    Lt = KR.kron_reduce(_lap(W), np.array([0, 2, 4]))
    g1 = 1.0 / (1.0 / w[0] + 1.0 / w[1])
    g2 = 1.0 / (1.0 / w[2] + 1.0 / w[3])
    want = np.array([[g1, -g1, 0.0], [-g1, g1 + g2, -g2], [0.0, -g2, g2]])
    assert np.allclose(Lt, want, rtol=0, atol=1e-14)


def test_star_mesh_closed_form():
    """Removing the centre of a star gives the complete graph with
    conductances w_i w_j / sum(w) (the star-mesh transform)."""
    w = np.array([0.3, 1.1, 2.0, 0.7, 1.6])
    N = len(w) + 1
    W = np.zeros((N, N))
    W[0, 1:] = W[1:, 0] = w
    Lt = KR.kron_reduce(_lap(W), np.arange(1, N))
    C = np.outer(w, w) / w.sum()
    np.fill_diagonal(C, 0.0)
    want = np.diag(C.sum(axis=1)) - C
    assert np.allclose(Lt, want, rtol=0, atol=1e-14)


def test_effective_resistance_preserved():
    """Effective resistances between kept nodes, from the pseudo-inverse of
    the full Laplacian, equal those of the reduced one."""
    rng = np.random.default_rng(0)
    N = 40
    L = _lap(_random_graph(N, rng)).toarray()
    omega = np.sort(rng.choice(N, 12, replace=False))
    Lt = KR.kron_reduce(L, omega)
    P, Pt = np.linalg.pinv(L), np.linalg.pinv(Lt)
    for a in range(len(omega)):
        for b in range(a + 1, len(omega)):
            i, j = omega[a], omega[b]
            r_full = P[i, i] + P[j, j] - 2 * P[i, j]
            r_red = Pt[a, a] + Pt[b, b] - 2 * Pt[a, b]
            assert r_red == pytest.approx(r_full, rel=1e-9)


@pytest.mark.parametrize("lap_type", [O.LAP_COMBINATORIAL, O.LAP_NORMALIZED])
def test_minimum_energy_by_least_squares(lap_type):
    """x_b^T L~ x_b = min over x_a of x^T L x, the minimum taken by a
    least-squares solve through the incidence factor L = G^T G."""
    rng = np.random.default_rng(1)
    N = 30
    W = _random_graph(N, rng)
    deg = W.sum(axis=1)
    s = np.sqrt(deg) if lap_type == O.LAP_NORMALIZED else np.ones(N)
    G = []
    for i in range(N):
        for j in range(i + 1, N):
            if W[i, j] > 0:
                g = np.zeros(N)
                g[i], g[j] = 1.0 / s[i], -1.0 / s[j]
                G.append(np.sqrt(W[i, j]) * g)
    G = np.array(G)
    omega = np.sort(rng.choice(N, 9, replace=False))
    abar = np.setdiff1d(np.arange(N), omega)
    Lt = KR.kron_reduce(_lap(W, lap_type), omega)
    for _ in range(3):
        xb = rng.standard_normal(len(omega))
        xa, *_ = np.linalg.lstsq(G[:, abar], -G[:, omega] @ xb, rcond=None)
        energy = np.sum((G[:, abar] @ xa + G[:, omega] @ xb) ** 2)
        assert xb @ Lt @ xb == pytest.approx(energy, rel=1e-10)


def test_quotient_two_steps_equal_one():
    rng = np.random.default_rng(2)
    N = 50
    L = _lap(_random_graph(N, rng), O.LAP_NORMALIZED)
    keep1 = np.sort(rng.choice(N, 25, replace=False))
    sub = np.sort(rng.choice(25, 10, replace=False))
    two = KR.kron_reduce(KR.kron_reduce(L, keep1), sub)
    one = KR.kron_reduce(L, keep1[sub])
    assert np.allclose(two, one, rtol=0, atol=1e-12)


@pytest.mark.parametrize("lap_type", [O.LAP_COMBINATORIAL, O.LAP_NORMALIZED])
def test_laplacian_invariants(lap_type):
    rng = np.random.default_rng(3)
    N = 60
    W = _random_graph(N, rng)
    omega = np.sort(rng.choice(N, 20, replace=False))
    Lt = KR.kron_reduce(_lap(W, lap_type), omega)
    assert np.allclose(Lt, Lt.T, rtol=0, atol=1e-13)
    off = Lt - np.diag(np.diag(Lt))
    assert off.max() <= 1e-14
    assert np.linalg.eigvalsh(Lt).min() >= -1e-12
    if lap_type == O.LAP_COMBINATORIAL:
        assert np.abs(Lt.sum(axis=1)).max() < 1e-12
    else:
        # L_n D^1/2 1 = 0, and the harmonic extension of its sampled part
        # is itself, so L~ (D^1/2 1)(omega) = 0
        v = np.sqrt(W.sum(axis=1))[omega]
        assert np.abs(Lt @ v).max() < 1e-12


def test_connectivity_through_unsampled_nodes():
    """Kept nodes i != j are coupled in L~ exactly when an edge joins them or
    a path joins them whose interior nodes are all unsampled."""
    rng = np.random.default_rng(4)
    N = 80
    W = np.zeros((N, N))
    for _ in range(70):  # sparse, several components
        i, j = rng.choice(N, 2, replace=False)
        W[i, j] = W[j, i] = rng.uniform(0.2, 1.0)
    adj = [np.flatnonzero(W[i]) for i in range(N)]
    ncomp, comp = csg.connected_components(sp.csr_matrix(W))
    omega = []
    for c in range(ncomp):  # every component gets a sampled node, then more
        omega.append(int(np.flatnonzero(comp == c)[0]))
    omega = np.unique(np.concatenate([omega, rng.choice(N, 20, replace=False)]))
    sampled = np.zeros(N, dtype=bool)
    sampled[omega] = True
    Lt = KR.kron_reduce(_lap(W), omega)
    for a, i in enumerate(omega):
        reach = set()
        seen = {int(i)}
        q = deque([int(i)])
        while q:
            u = q.popleft()
            for v in adj[u]:
                v = int(v)
                if sampled[v]:
                    reach.add(v)
                elif v not in seen:
                    seen.add(v)
                    q.append(v)
        for b, j in enumerate(omega):
            if a != b:
                assert (abs(Lt[a, b]) > 1e-15) == (int(j) in reach)


def test_full_sampling_is_identity_map():
    rng = np.random.default_rng(5)
    L = _lap(_random_graph(20, rng), O.LAP_NORMALIZED)
    assert np.array_equal(KR.kron_reduce(L, np.arange(20)), L.toarray())


def test_component_without_sample_rejected():
    W = np.zeros((6, 6))
    W[0, 1] = W[1, 0] = 1.0
    W[2, 3] = W[3, 2] = W[3, 4] = W[4, 3] = 0.5
    with pytest.raises(ValueError):
        KR.kron_reduce(_lap(W), np.array([0, 5]))  # component {2, 3, 4} unsampled


def test_csr_form_holds_every_entry():
    rng = np.random.default_rng(6)
    L = _lap(_random_graph(25, rng), O.LAP_NORMALIZED)
    om = np.sort(rng.choice(25, 8, replace=False))
    C = KR.kron_reduce_csr(L, om)
    assert C.nnz == 64 and np.array_equal(C.toarray(), KR.kron_reduce(L, om))
