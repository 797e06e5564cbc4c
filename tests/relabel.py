"""Test helper: the oracle run on the dealt relabeling of an instance.

With interleave on, the GPU's tiled schedule works on internal labels:
caller object i gets label lab(i), dealt in rounds over the blocks of B
(round r gives the next object to every block with more than r slots).  That
is the tiled schedule applied to the relabeled instance, so the oracle runs
schedule 2 on the relabeled instance and its state is mapped back to the
caller's labels here.  Written independently of the library."""
import itertools

import numpy as np

import oracle


def deal_labels(n, B):
    nb = -(-n // B)
    lab = np.empty(n, dtype=np.int64)
    i = 0
    for r in range(B):
        for b in range(nb):
            if min(B, n - b * B) > r:
                lab[i] = b * B + r
                i += 1
    assert i == n and len(set(lab.tolist())) == n
    return lab


def _pidx(n, i, j):
    return i * n - i * (i + 1) // 2 + (j - i - 1)


def _c2(m):
    return np.where(m >= 2, m * (m - 1) // 2, 0)


def _c3(m):
    return np.where(m >= 3, m * (m - 1) * (m - 2) // 6, 0)


class RelabeledOracle:
    def __init__(self, n, d, w, eps, B):
        self.n, self.B = n, B
        self.lab = deal_labels(n, B)
        iu, ju = np.triu_indices(n, 1)
        a, b = self.lab[iu], self.lab[ju]
        self.pmap = _pidx(n, np.minimum(a, b), np.maximum(a, b))   # caller pair -> internal pair
        P = len(d)
        dint, wint = np.empty(P), np.empty(P)
        dint[self.pmap] = d
        wint[self.pmap] = w
        self.st = oracle.State(n, dint, wint, eps)
        T = list(itertools.combinations(range(n), 3))
        t = np.array(T, dtype=np.int64).reshape(-1, 3)
        la, lb, lc = self.lab[t[:, 0]], self.lab[t[:, 1]], self.lab[t[:, 2]]
        lo = np.minimum(la, np.minimum(lb, lc))
        hi = np.maximum(la, np.maximum(lb, lc))
        mid = la + lb + lc - lo - hi
        rank = (_c3(n) - _c3(n - lo)) + (_c2(n - 1 - lo) - _c2(n - mid)) + (hi - mid - 1)

        def out(third):   # internal row that leaves `third` out
            return np.where(third == hi, 0, np.where(third == mid, 1, 2))

        rows = np.stack([out(lc), out(lb), out(la)], 1)            # caller rows ij, ik, jk
        self.tmap = 3 * rank[:, None] + rows                        # caller (triplet, row) -> internal

    def sweep(self, k=1):
        for _ in range(k):
            self.st.sweep(2, self.B)

    @property
    def x(self):
        return self.st.x[self.pmap]

    @property
    def f(self):
        return self.st.f[self.pmap]

    @property
    def ytri(self):
        return self.st.ytri[self.tmap].reshape(-1)

    @property
    def ypair(self):
        return np.stack([self.st.ypair[2 * self.pmap], self.st.ypair[2 * self.pmap + 1]], 1).reshape(-1)

    def max_violation(self):
        return self.st.max_violation()

    def objectives(self):
        return self.st.objectives()
