"""Pins of the SCFV oracle (CPU): the PCA projection on its basis rows, the
joint log-likelihood against scipy's
multivariate normal, both Fisher gradients against finite differences of the
GMM log-likelihood, a one-component model against its closed form, the
paper's matrix form of the distance (Eq. 10) against the direct sum with V
the variance, delta against numpy's std, and the ranking and bits by hand."""
import math
import os

import numpy as np
import pytest
from scipy.stats import multivariate_normal

from oracle import scfv_oracle as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_model(seed, n_comp=6, dim=4, n_in=10):
    rng = np.random.default_rng(seed)
    P = np.linalg.qr(rng.normal(size=(n_in, dim)))[0].T
    w = rng.random(n_comp) + 0.2
    return {"pca_mean": rng.normal(0, 0.1, n_in), "pca": P, "weights": w / w.sum(),
            "means": rng.normal(0, 0.6, (n_comp, dim)), "variances": rng.uniform(0.2, 0.8, (n_comp, dim))}


def _loglik(X, m):
    Y = S.pca(X, m["pca_mean"], m["pca"])
    l = S.log_joint(Y, m["weights"], m["means"], m["variances"])
    mx = l.max(axis=1, keepdims=True)
    return float((mx[:, 0] + np.log(np.exp(l - mx).sum(axis=1))).sum())


def test_pca_projects_onto_the_basis_rows():
    """The projection is onto the rows of the orthonormal basis after the mean
    is taken off: mean + 2.5 P[j] maps to 2.5 e_j, the mean itself to 0, and a
    vector orthogonal to every row to 0."""
    m = _small_model(8)
    P, mean = m["pca"], m["pca_mean"]
    for j in range(4):
        np.testing.assert_allclose(S.pca((mean + 2.5 * P[j])[None], mean, P)[0], 2.5 * np.eye(4)[j], atol=1e-12)
    np.testing.assert_allclose(S.pca(mean[None], mean, P), 0.0, atol=1e-12)
    v = np.random.default_rng(9).normal(size=10)
    v -= P.T @ (P @ v)                      # remove the basis components
    np.testing.assert_allclose(S.pca((mean + v)[None], mean, P), 0.0, atol=1e-12)


def test_log_joint_matches_scipy():
    m = _small_model(1)
    Y = np.random.default_rng(2).normal(size=(7, 4))
    l = S.log_joint(Y, m["weights"], m["means"], m["variances"])
    for i in range(6):
        ref = np.log(m["weights"][i]) + multivariate_normal(m["means"][i], np.diag(m["variances"][i])).logpdf(Y)
        np.testing.assert_allclose(l[:, i], ref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(S.posteriors(Y, m["weights"], m["means"], m["variances"]).sum(axis=1), 1.0, rtol=1e-12)


@pytest.mark.parametrize("which", ["mu", "sigma"])
def test_gradients_match_finite_differences(which):
    m = _small_model(3)
    X = np.random.default_rng(4).normal(0, 0.5, (9, 10))
    g_mu, g_sig, _ = S.fisher(X, m)
    K, h = len(X), 1e-6
    for i in range(6):
        for k in range(4):
            mp = {kk: np.array(v, copy=True) for kk, v in m.items()}
            mm = {kk: np.array(v, copy=True) for kk, v in m.items()}
            if which == "mu":
                mp["means"][i, k] += h
                mm["means"][i, k] -= h
                dL = (_loglik(X, mp) - _loglik(X, mm)) / (2 * h)          # sum_t gamma (y - mu) / v
                want = math.sqrt(m["variances"][i, k]) * dL / (K * math.sqrt(m["weights"][i]))
                got = g_mu[i, k]
            else:
                s = math.sqrt(m["variances"][i, k])
                mp["variances"][i, k] = (s + h) ** 2
                mm["variances"][i, k] = (s - h) ** 2
                dL = (_loglik(X, mp) - _loglik(X, mm)) / (2 * h)          # d/ds: sum_t gamma ((y-mu)^2/s^3 - 1/s)
                want = s * dL / (K * math.sqrt(2 * m["weights"][i]))
                got = g_sig[i, k]
            assert abs(got - want) <= 1e-6 * max(1.0, abs(want)), (which, i, k, got, want)


def test_one_component_closed_form():
    m = _small_model(5, n_comp=1)
    m["weights"] = np.array([1.0])
    X = np.random.default_rng(6).normal(0, 0.5, (13, 10))
    g_mu, g_sig, delta = S.fisher(X, m)
    Y = S.pca(X, m["pca_mean"], m["pca"])
    z = (Y - m["means"][0]) / np.sqrt(m["variances"][0])
    np.testing.assert_allclose(g_mu[0], z.mean(axis=0), rtol=1e-12)
    np.testing.assert_allclose(g_sig[0], (z * z - 1).mean(axis=0) / math.sqrt(2), rtol=1e-12)
    assert delta[0] == pytest.approx(np.std(g_mu[0]))


def test_matrix_form_of_the_distance():
    """Eq. 10: P = (D.*D)(1./V)^T - 2 D (M./V)^T + O ((M.*M)./V)^T equals
    sum_k (D_ik - M_jk)^2 / V_jk when V holds the variances."""
    rng = np.random.default_rng(7)
    D, M, V = rng.normal(size=(11, 32)), rng.normal(size=(20, 32)), rng.uniform(0.1, 2, (20, 32))
    P = (D * D) @ (1 / V).T - 2 * D @ (M / V).T + np.ones_like(D) @ ((M * M) / V).T
    direct = np.array([[((D[i] - M[j]) ** 2 / V[j]).sum() for j in range(20)] for i in range(11)])
    np.testing.assert_allclose(P, direct, rtol=1e-10, atol=1e-10)
    l = S.log_joint(D, np.full(20, 1 / 20), M, V)
    np.testing.assert_allclose(-2 * (l - np.log(1 / 20)) - np.log(2 * np.pi * V).sum(axis=1), direct, rtol=1e-10)


def test_ranking_bits_and_empty_image():
    d = np.array([0.5, 2.0, 0.5, 1.0])
    np.testing.assert_array_equal(S.ranking(d), [1, 3, 0, 2])
    g = np.zeros((4, 32))
    g[1, [0, 5, 31]] = 1.0
    g[3, 2] = -1.0
    np.testing.assert_array_equal(S.sign_bits(g, S.ranking(d), 2), [1 | 32 | (1 << 31), 0])
    model = dict(np.load(os.path.join(GOLDEN, "scfv_model.npz")))
    g_mu, g_sig, delta = S.fisher(np.zeros((0, 128)), model)
    assert not g_mu.any() and not g_sig.any() and not delta.any()
    np.testing.assert_array_equal(S.ranking(delta), np.arange(512))


def test_stand_in_model_is_a_valid_gmm():
    m = np.load(os.path.join(GOLDEN, "scfv_model.npz"))
    P = m["pca"].astype(np.float64)
    np.testing.assert_allclose(P @ P.T, np.eye(32), atol=1e-5)
    assert m["means"].shape == (512, 32) and (m["variances"] > 0).all()
    assert abs(m["weights"].sum() - 1) < 1e-5
