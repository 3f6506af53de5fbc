"""Closed-form and quadrature evidences used to pin the checker and the GPU path.

Each function restates a textbook integral with library special functions; none
calls the sampler.
"""
import numpy as np
from scipy import integrate, special, stats


def box_gauss_logZ(mu, sigma, a, b):
    """Uniform prior on the box [a, b], normalised isotropic Gaussian likelihood:
    Z = prod_i [Phi((b_i-mu_i)/s) - Phi((a_i-mu_i)/s)] / prod_i (b_i - a_i)."""
    mu, a, b = map(np.asarray, (mu, a, b))
    mass = special.log_ndtr((b - mu) / sigma)
    lo = special.log_ndtr((a - mu) / sigma)
    # log(Phi(hi) - Phi(lo)) computed as log Phi(hi) + log1p(-exp(lo - hi))
    return float(np.sum(mass + np.log1p(-np.exp(lo - mass))) - np.sum(np.log(b - a)))


def box_gmm_logZ(mus, sigma, a, b):
    """Equal-weight mixture of normalised isotropic Gaussians under a uniform box prior."""
    terms = [box_gauss_logZ(m, sigma, a, b) for m in np.atleast_2d(mus)]
    return float(special.logsumexp(terms) - np.log(len(terms)))


def gauss_gauss_logZ(mu, sigma, m0, s0):
    """Prior N(m0, s0^2 I), normalised likelihood N(x; mu, sigma^2 I):
    Z = N(mu; m0, (s0^2 + sigma^2) I)."""
    mu, m0, s0 = map(np.asarray, (mu, m0, s0))
    var = s0 ** 2 + sigma ** 2
    return float(np.sum(stats.norm.logpdf(mu, loc=m0, scale=np.sqrt(var))))


def rastrigin_logZ(alpha, d, r=5.14, A=10.0):
    """Semi-analytic evidence of the Gaussian/Rastrigin mixture on [-r, r]^d
    (App. F.3): one-dimensional integrals by adaptive quadrature."""
    i1, _ = integrate.quad(lambda x: np.exp(-0.5 * x * x), -r, r, limit=200)
    i2, _ = integrate.quad(lambda x: np.exp(A * np.cos(2 * np.pi * x) - A), -r, r, limit=400)
    t1 = np.log(alpha) + d * np.log(i1) if alpha > 0 else -np.inf
    t2 = np.log1p(-alpha) + d * np.log(i2) if alpha < 1 else -np.inf
    return float(np.logaddexp(t1, t2) - d * np.log(2 * r))


def gp_quadrature_logZ(loglik, a, b, panels=8, order=6):
    """Evidence of a 3-parameter likelihood under a uniform box prior by
    composite Gauss-Legendre quadrature (panels x order nodes per axis):
    Z = (1/vol) int_box L(theta) d theta, evaluated in log space."""
    xq, wq = np.polynomial.legendre.leggauss(order)
    axes = []
    for lo, hi in zip(a, b):
        edges = np.linspace(lo, hi, panels + 1)
        pts = np.concatenate([(e0 + e1) / 2 + (e1 - e0) / 2 * xq for e0, e1 in zip(edges[:-1], edges[1:])])
        wts = np.concatenate([(e1 - e0) / 2 * wq for e0, e1 in zip(edges[:-1], edges[1:])])
        axes.append((pts, wts))
    lv = []
    lw = []
    for p0, w0 in zip(*axes[0]):
        for p1, w1 in zip(*axes[1]):
            for p2, w2 in zip(*axes[2]):
                lv.append(loglik(np.array([p0, p1, p2])))
                lw.append(np.log(w0 * w1 * w2))
    lv, lw = np.array(lv), np.array(lw)
    vol = np.prod(np.asarray(b) - np.asarray(a))
    return float(special.logsumexp(lv + lw) - np.log(vol))
