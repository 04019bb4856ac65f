"""Chebyshev filter polynomial for the oracle (test infrastructure only).

Section 2 of the paper: polynomial filtering uses a low-order polynomial
P(K) approximating K^-1, built from Chebyshev polynomials, with the order p
as its only parameter.  The paper does not print the construction.
Reading: the relative-error minimax approximation of 1/x on [eps, lam],

    x P(x) = 1 - R(x),   R(x) = T_{n+1}((mu - x)/nu) / T_{n+1}(mu/nu),
    mu = (lam + eps)/2,  nu = (lam - eps)/2,

so |1 - x P(x)| <= 1 / T_{n+1}(mu/nu) on [eps, lam].  Its roots are

    z_k = mu (1 - cos t_k) - i sqrt(eps lam) sin t_k,  t_k = 2 pi k/(n+1),
    k = 1..n,

and P(x) = c prod_k (x - z_k) with c = 2^n (-1)^n / (nu^{n+1} T_{n+1}(mu/nu)).
(z_k and z_{n+1-k} are conjugate; for even n, P > 0 on (0, inf).)  The
closed form R(x) is evaluated with numpy's Chebyshev basis; the oracle
applies P(K) to a vector as the plain root product, with conjugate roots
paired into real quadratics.
"""
import numpy as np
from numpy.polynomial import chebyshev as C


class ChebyshevFilter:
    def __init__(self, n, eps, lam):
        self.n, self.eps, self.lam = int(n), float(eps), float(lam)
        self.mu = 0.5 * (self.lam + self.eps)
        self.nu = 0.5 * (self.lam - self.eps)
        self.y0 = self.mu / self.nu
        self._tn1 = C.Chebyshev.basis(self.n + 1)

    # closed forms --------------------------------------------------------
    def R(self, x):
        return self._tn1((self.mu - np.asarray(x)) / self.nu) / self._tn1(self.y0)

    def value(self, x):
        """P(x) = (1 - R(x)) / x."""
        x = np.asarray(x, dtype=np.float64)
        return (1.0 - self.R(x)) / x

    def error_bound(self):
        return 1.0 / self._tn1(self.y0)

    # factored form -------------------------------------------------------
    def roots(self):
        k = np.arange(1, self.n + 1)
        th = 2 * np.pi * k / (self.n + 1)
        return self.mu * (1 - np.cos(th)) - 1j * np.sqrt(self.eps * self.lam) * np.sin(th)

    def scale(self):
        return 2.0 ** self.n * (-1) ** self.n / (self.nu ** (self.n + 1) * self._tn1(self.y0))

    def value_product(self, x):
        x = np.asarray(x, dtype=np.complex128)
        out = self.scale() * np.ones_like(x)
        for z in self.roots():
            out = out * (x - z)
        return out

    # operator application -------------------------------------------------
    def apply(self, K, v):
        """P(K) v as c prod_k (K - z_k) v (even n), conjugate roots applied as
        the real quadratics K^2 - 2 Re(z_k) K + |z_k|^2, c spread evenly over them."""
        assert self.n % 2 == 0, "the filter is used with even degree only"
        m = self.n // 2
        if m == 0:
            return self.scale() * v
        z = self.roots()
        f = self.scale() ** (1.0 / m)
        out = v
        for k in range(m):
            a, b = 2 * z[k].real, abs(z[k]) ** 2
            Kv = K(out)
            out = f * (K(Kv) - a * Kv + b * out)
        return out

    def apply_half(self, K, v, dagger=False):
        """C(K) v with C = sqrt(c) prod_{k<=n/2} (K - z_k), so that C^dag C = P (even n).

        dagger=True applies C^dag = sqrt(c) prod (K - conj z_k)."""
        assert self.n % 2 == 0
        z = self.roots()[: self.n // 2]
        if dagger:
            z = z.conj()
        out = np.sqrt(self.scale()) * v
        for zk in z:
            out = K(out) - zk * out
        return out

    def roots_times_x(self):
        """Roots of x P(x): {0} and z_k, with the same scale c."""
        return np.concatenate([[0.0 + 0.0j], self.roots()])


class RatioFilter:
    """Q = P_hi / P_lo for two filters on the same [eps, lam] (Section 3.3 of the
    paper, two-filter action S_2PF, "Q(K) = P_2(K)/P_1(K)").  Q is a polynomial when
    every root of P_lo is a root of P_hi, which for the reading above holds when
    (n_lo + 1) divides (n_hi + 1); its roots are the remaining roots of P_hi and its
    scale c_hi / c_lo.  Applied, like the filter, as the root product with conjugate
    roots paired into real quadratics."""

    def __init__(self, hi, lo):
        assert hi.eps == lo.eps and hi.lam == lo.lam and (hi.n + 1) % (lo.n + 1) == 0
        self.hi, self.lo = hi, lo
        zl = lo.roots()
        keep = [z for z in hi.roots() if np.min(np.abs(zl - z)) > 1e-9 * hi.lam]
        self._roots = np.array(keep)
        assert len(self._roots) == hi.n - lo.n
        self.n = len(self._roots)

    def roots(self):
        return self._roots

    def scale(self):
        return self.hi.scale() / self.lo.scale()

    def value(self, x):
        return self.hi.value(x) / self.lo.value(x)

    def value_product(self, x):
        out = self.scale() * np.ones_like(np.asarray(x, dtype=np.complex128))
        for z in self._roots:
            out = out * (x - z)
        return out

    def _pairs(self):
        """Indices pairing each root with its conjugate."""
        z = self._roots
        used, pairs = set(), []
        for i in range(len(z)):
            if i in used:
                continue
            j = int(np.argmin(np.abs(z - z[i].conj()) + np.where(np.arange(len(z)) == i, np.inf, 0)))
            used.update((i, j))
            pairs.append((i, j))
        return pairs

    def apply(self, K, v):
        pairs = self._pairs()
        f = self.scale() ** (1.0 / len(pairs))
        out = v
        for i, _ in pairs:
            zi = self._roots[i]
            Kv = K(out)
            out = f * (K(Kv) - 2 * zi.real * Kv + abs(zi) ** 2 * out)
        return out

    def apply_half(self, K, v, dagger=False):
        """D v with D = sqrt(scale) prod over one root of each conjugate pair, D^dag D = Q."""
        z = np.array([self._roots[i] for i, _ in self._pairs()])
        if dagger:
            z = z.conj()
        out = np.sqrt(self.scale()) * v
        for zk in z:
            out = K(out) - zk * out
        return out
