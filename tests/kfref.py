"""Batch maximum-a-posteriori solution of the linear track model in float64.

A Kalman filter on a linear-Gaussian state-space model returns, after each
update, the mean and covariance of the state given the prior and all
measurements so far -- the same quantities as the weighted least-squares
problem over the initial state and the process-noise terms (textbook
equivalence of recursive and batch least squares).  This module solves that
batch problem with numpy.linalg.lstsq, independently of the oracle's
recursive arithmetic, for one block of the model:
  state_k = F(dx_k) state_{k-1} + w_k e_slope,  w_k ~ N(0, q |dx_k|)
  meas_k  = state_k[0] + v_k,                   v_k ~ N(0, r)
"""
from __future__ import annotations

import numpy as np


def f_matrix(dim: int, dx: float) -> np.ndarray:
    if dim == 3:
        return np.array([[1.0, dx, 0.5 * dx * dx], [0.0, 1.0, dx], [0.0, 0.0, 1.0]])
    return np.array([[1.0, dx], [0.0, 1.0]])


def batch_filter(m0, p0_diag, xs, meas, r, q):
    """Filtered means/covariances after each measurement k = 1..n-1 and the
    one-step predictions of meas for k = 1..n-1.

    m0, p0_diag: prior mean and diagonal covariance at xs[0];
    xs: reference x of every step; meas: measurement at every step (meas[0]
    unused: it is part of the prior)."""
    dim = len(m0)
    n = len(xs)
    preds = np.zeros(n)
    means = np.zeros((n, dim))
    covs = np.zeros((n, dim, dim))
    means[0] = m0
    covs[0] = np.diag(p0_diag)
    for k in range(1, n):
        # unknowns: x0 (dim), w_1..w_k (k)
        nu = dim + k
        maps = []  # linear map unknowns -> state_i (dim x nu)
        a = np.zeros((dim, nu))
        a[:, :dim] = np.eye(dim)
        for i in range(1, k + 1):
            fm = f_matrix(dim, xs[i] - xs[i - 1])
            a = fm @ a
            a[1, dim + i - 1] += 1.0
            maps.append(a.copy())
        rows, rhs = [], []
        for d in range(dim):
            e = np.zeros(nu)
            e[d] = 1.0 / np.sqrt(p0_diag[d])
            rows.append(e)
            rhs.append(m0[d] / np.sqrt(p0_diag[d]))
        for i in range(1, k + 1):
            qi = q * abs(xs[i] - xs[i - 1])
            e = np.zeros(nu)
            if qi > 0:
                e[dim + i - 1] = 1.0 / np.sqrt(qi)
            else:
                e[dim + i - 1] = 1e12  # pins w_i to zero
            rows.append(e)
            rhs.append(0.0)
        for i in range(1, k + 1):
            rows.append(maps[i - 1][0] / np.sqrt(r))
            rhs.append(meas[i] / np.sqrt(r))
        jm = np.array(rows)
        sol, *_ = np.linalg.lstsq(jm, np.array(rhs), rcond=None)
        amap = maps[k - 1]
        means[k] = amap @ sol
        cov_u = np.linalg.inv(jm.T @ jm)
        covs[k] = amap @ cov_u @ amap.T
        # prediction of step k from the data up to k-1
        if k == 1:
            prev_mean = np.asarray(m0, float)
        else:
            prev_mean = means[k - 1]
        preds[k] = (f_matrix(dim, xs[k] - xs[k - 1]) @ prev_mean)[0]
    return preds, means, covs
