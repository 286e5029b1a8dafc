"""FP64 oracle of the SCFV aggregation (the global descriptor of Sec. III-D
and its matrix form in Sec. IV-C).

TEST INFRASTRUCTURE ONLY: the tests are the only users.

For the K local descriptors x_t (128-D) of one image:

    y_t = P (x_t - m)                                    PCA to 32 dimensions
    l_t(i) = log w_i - 1/2 sum_k [ (y_tk - mu_ik)^2 / v_ik + log(2 pi v_ik) ]
    gamma_t(i) = exp(l_t(i)) / sum_j exp(l_t(j))          posterior, Eq. 6
    g_mu(i)    = 1 / (K sqrt(w_i))     sum_t gamma_t(i) (y_t - mu_i) / s_i                 Eq. 7
    g_sigma(i) = 1 / (K sqrt(2 w_i))   sum_t gamma_t(i) ((y_t - mu_i)^2 / v_i - 1)
    delta(i)   = population standard deviation of the 32 entries of g_mu(i)              Eq. 8

with v_i the diagonal variances and s_i = sqrt(v_i).  Components are ranked
by delta descending, ties to the lower index; the selected components' sign
bits (bit k set when g_mu(i)_k > 0) form the binary descriptor.

Readings where the paper is loose: in the distance of Eq. 9 the divisor V is
the variance (so the matrix form of Eq. 10 is the same sum); Eq. 7 divides by
the standard deviation, as the Fisher score does; the variance gradient is
the Fisher score of the standard deviation (Eq. 13), which the matrix form of Eq. 14
computes; K is the number of the image's descriptors, and an image with none
gives zero gradients.
"""
from __future__ import annotations

import math

import numpy as np

N_COMP, DIM = 512, 32


def pca(X, mean, P):
    return (np.asarray(X, np.float64) - np.asarray(mean, np.float64)) @ np.asarray(P, np.float64).T


def log_joint(Y, w, means, var):
    """l[t, i] = log w_i + log N(y_t; mu_i, diag(v_i))."""
    Y, means, var = (np.asarray(a, np.float64) for a in (Y, means, var))
    l = np.empty((len(Y), len(w)))
    for i in range(len(w)):
        d = Y - means[i]
        l[:, i] = math.log(w[i]) - 0.5 * ((d * d / var[i]).sum(axis=1) + np.log(2 * math.pi * var[i]).sum())
    return l


def posteriors(Y, w, means, var):
    l = log_joint(Y, w, means, var)
    m = l.max(axis=1, keepdims=True)
    e = np.exp(l - m)
    return e / e.sum(axis=1, keepdims=True)


def fisher(X, model):
    """(g_mu, g_sigma, delta) of one image's descriptors X (K x 128)."""
    w = np.asarray(model["weights"], np.float64)
    means = np.asarray(model["means"], np.float64)
    var = np.asarray(model["variances"], np.float64)
    g_mu = np.zeros((len(w), means.shape[1]))
    g_sig = np.zeros_like(g_mu)
    K = len(X)
    if K:
        Y = pca(X, model["pca_mean"], model["pca"])
        gam = posteriors(Y, w, means, var)
        sd = np.sqrt(var)
        for i in range(len(w)):
            d = (Y - means[i]) / sd[i]
            g_mu[i] = (gam[:, i:i + 1] * d).sum(axis=0) / (K * math.sqrt(w[i]))
            g_sig[i] = (gam[:, i:i + 1] * (d * d - 1.0)).sum(axis=0) / (K * math.sqrt(2.0 * w[i]))
    delta = np.sqrt(((g_mu - g_mu.mean(axis=1, keepdims=True)) ** 2).mean(axis=1))
    return g_mu, g_sig, delta


def ranking(delta):
    """Component indices by delta descending, ties to the lower index."""
    return np.array(sorted(range(len(delta)), key=lambda i: (-delta[i], i)), np.int32)


def sign_bits(g_mu, order, n_select):
    """uint32 per selected component in rank order: bit k = g_mu[i, k] > 0."""
    out = np.zeros(n_select, np.uint32)
    for r in range(n_select):
        i = order[r]
        word = 0
        for k in range(g_mu.shape[1]):
            if g_mu[i, k] > 0:
                word |= 1 << k
        out[r] = word
    return out
