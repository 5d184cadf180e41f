"""FP64 reference of the divide-and-conquer (bridging) pathwise sampler.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package; the product path never does.

Section 2.4.2 (divide-and-conquer approach) and Appendix A.2.3. Given the
filtering moments (m^f_t, P^f_t) of the LGSSM, the smoothing law of the path
is sampled top-down through bridging conditionals p(x_l | x_k, x_m, y):

  * leaves (Appendix A.2.3, initialisation of the tree): for t = 0 .. T-2,
        E_{t:t+1} = P^f_t F_t^T (F_t P^f_t F_t^T + Q_t)^{-1},
        g_{t:t+1} = m^f_t - E_{t:t+1} (F_t m^f_t + b_t),
        L_{t:t+1} = P^f_t - E_{t:t+1} F_t P^f_t,
    so that p(x_t | x_{t+1}, y) = N(E x_{t+1} + g, L);
  * composition of adjacent intervals k < l < m (the (E, g, L) rule):
        E_{k:m} = E_{k:l} E_{l:m},  g_{k:m} = E_{k:l} g_{l:m} + g_{k:l},
        L_{k:m} = E_{k:l} L_{l:m} E_{k:l}^T + L_{k:l};
  * the bridge of the split point l (the (G, Gamma, w, V) rule):
        G = L_{l:m} E_{k:l}^T L_{k:m}^{-1},  Gamma = E_{l:m} - G E_{k:m},
        w = g_{l:m} - G g_{k:m},            V = L_{l:m} - G L_{k:m} G^T,
    so that p(x_l | x_k, x_m, y) = N(G x_k + Gamma x_m + w, V);
  * sampling: x_{T-1} ~ N(m^f_{T-1}, P^f_{T-1}), then x_0 | x_{T-1} from the
    root's (E, g, L), then the split points level by level from the root
    down, all split points of one level in parallel.

The tree is the dyadic one that the appendix builds bottom-up (intervals
[t, t+1], then [2a, 2a+2], then [4a, 4a+4], ...): with n = T - 1 unit
intervals, node a of level j covers [a 2^j, min((a+1) 2^j, n)] and splits at
l = (2a+1) 2^(j-1) when l < n; a node whose right half is empty is its left
child unchanged. For n a power of two the split points are the midpoints of
the main text's recursion. Noise: x_t uses eps_t (the t-th row of eps) for
every t, whichever level samples it.

parity pins (tests/test_oracle_bridging.py): every node's (E, g, L) and
bridge equal the conditionals of the dense smoothing Gaussian of the stacked
path; the sampler's affine map eps -> x has the dense smoothing mean and
covariance; T = 2 reproduces the RTS sampler.
"""
import numpy as np


def _at(arr, t, ndim):
    arr = np.asarray(arr, dtype=np.float64)
    return arr if arr.ndim == ndim else arr[t]


def _sym(a):
    return 0.5 * (a + a.T)


def leaf_elements(kf, F, b, Q):
    """(E, g, L) of the unit intervals [t, t+1], t = 0 .. T-2."""
    mf, Pf = kf["mf"], kf["Pf"]
    T = mf.shape[0]
    out = []
    for t in range(T - 1):
        Ft, bt, Qt = _at(F, t, 2), _at(b, t, 1), _at(Q, t, 2)
        Pp = Ft @ Pf[t] @ Ft.T + Qt
        E = np.linalg.solve(Pp, Ft @ Pf[t]).T          # P^f F^T Pp^{-1} (Pp symmetric)
        g = mf[t] - E @ (Ft @ mf[t] + bt)
        L = _sym(Pf[t] - E @ Ft @ Pf[t])
        out.append(dict(k=t, m=t + 1, l=None, E=E, g=g, L=L))
    return out


def compose(left, right):
    """(E, g, L) of [k, m] from those of [k, l] (left) and [l, m] (right)."""
    E = left["E"] @ right["E"]
    g = left["E"] @ right["g"] + left["g"]
    L = _sym(left["E"] @ right["L"] @ left["E"].T + left["L"])
    return dict(k=left["k"], m=right["m"], l=left["m"], E=E, g=g, L=L)


def bridge(left, right, node):
    """(G, Gamma, w, V) of p(x_l | x_k, x_m, y) for node = compose(left, right)."""
    G = np.linalg.solve(node["L"], left["E"] @ right["L"]).T    # L_{l:m} E_{k:l}^T L_{k:m}^{-1}
    Gam = right["E"] - G @ node["E"]
    w = right["g"] - G @ node["g"]
    V = _sym(right["L"] - G @ node["L"] @ G.T)
    return dict(G=G, Gam=Gam, w=w, V=V)


def build_tree(kf, F, b, Q):
    """Levels of the dyadic tree, leaves first; each node a dict with its
    interval (k, l, m) (l None where the node has one child), (E, g, L) and,
    where l is set, the bridge (G, Gam, w, V)."""
    levels = [leaf_elements(kf, F, b, Q)]
    while len(levels[-1]) > 1:
        prev = levels[-1]
        cur = []
        for a in range(0, len(prev), 2):
            if a + 1 < len(prev):
                node = compose(prev[a], prev[a + 1])
                node.update(bridge(prev[a], prev[a + 1], node))
            else:
                node = dict(prev[a])
                node["l"] = None
                for key in ("G", "Gam", "w", "V"):
                    node.pop(key, None)
            cur.append(node)
        levels.append(cur)
    return levels


def dnc_sample(kf, F, b, Q, eps):
    """One draw of x_{0:T-1} | y by the divide-and-conquer sampler, driven by eps [T, d]."""
    mf, Pf = kf["mf"], kf["Pf"]
    T, d = mf.shape
    x = np.full((T, d), np.nan)
    x[T - 1] = mf[T - 1] + np.linalg.cholesky(Pf[T - 1]) @ eps[T - 1]
    if T == 1:
        return x
    levels = build_tree(kf, F, b, Q)
    root = levels[-1][0]
    x[0] = root["E"] @ x[T - 1] + root["g"] + np.linalg.cholesky(root["L"]) @ eps[0]
    for level in reversed(levels[1:]):
        for node in level:                     # independent given the level above
            if node["l"] is None:
                continue
            k, l, m = node["k"], node["l"], node["m"]
            mean = node["G"] @ x[k] + node["Gam"] @ x[m] + node["w"]
            x[l] = mean + np.linalg.cholesky(node["V"]) @ eps[l]
    return x
