"""Block-splitting ADMM over an explicit random feature matrix, float64.

Test infrastructure (see the package header): never imported by the product.

Problem (Sec. 2.2, eq. (problem_linear), rewritten over blocks as eq. (prob2)):
    minimise  sum_i V(y_i, W^T z_i) + n lam r(W)
over W (D x m), with Z = [Z_ij] split into R row blocks and C column blocks.

Updates (Sec. 3, the Parikh-Boyd block-splitting equations around eq. (gp)),
all variables starting at zero, i = 1..R, j = 1..C:
  O_i    <- prox_{(1/rho) V}[Obar_i - nu_i]
  W_j    <- prox_{(n lam/rho) r}[Wbar_j - mu_j]
  (O_ij, What_ij) <- proj_{Z_ij}[Obar_ij + nu_i, Wbar_j - mu_ij]          eq. (gp)
         i.e. What_ij = (Z_ij^T Z_ij + I)^-1 [Wbar_j - mu_ij + Z_ij^T (Obar_ij + nu_i)]
              O_ij    = Z_ij What_ij                             eq. (gpWij), (gpOij)
  Wbar_j <- (W_j + sum_i What_ij) / (R + 1)
  Obar_ij <- O_ij + (O_i - sum_j O_ij) / (C + 1)                         eq. (obar_ij)
  Obar_i <- sum_j Obar_ij                                                eq. (obar)
  mu_j += W_j - Wbar_j ;  mu_ij += What_ij - Wbar_j ;  nu_i += O_i - Obar_i

Readings (the paper is silent or inconsistent; each is stated here once):
1. The update equations are authoritative.  The printed pseudo-code
   (Algorithm 1) drops the Z^T nu term from the graph-projection right-hand side
   and updates mu', mu with the previous Wbar; run literally it does not reach
   the minimiser (``variant="algorithm1_literal"`` reproduces it for the tests).
2. rho is the penalty of the SUM-scaled objective above ("sum"): the loss prox
   step is 1/rho and the regulariser prox step n lam / rho.  The paper's own
   l_i carries 1/n ("mean"), which is the same method with rho_paper = rho / n;
   ``rho_scale="mean"`` takes rho literally in that scaling.
3. The cache (eq. (cache)) is set up before the first graph projection.
4. Graph-projection form per block: (I + Z^T Z) when s_j <= n_i, otherwise the
   n_i x n_i form with (I + Z Z^T) (the remark after eq. (graphV)); both give the
   same projection and ``graph_projection`` implements both.

Variants: "equation" keeps every Obar_ij as printed; "reorganised" follows the
memory-efficient rewrite of Sec. 3 (U_ij = Z_ij^T O_ij, one Delta_i,
Z_ij^T Obar_ij = U_ij + Z_ij^T Delta_i / (C + 1),
Obar_i = sum_j O_ij / (C + 1) + C/(C + 1) O_i), with the Z^T nu term restored;
"incremental" is the equation form with each graph projection taken from the block's
previous (What_ij, O_ij): the projection is linear and fixes every point of the graph
(O_ij = Z_ij What_ij), so proj[Obar_ij + nu_i, Wbar_j - mu_ij] = (O_ij, What_ij) +
proj[Obar_ij + nu_i - O_ij, Wbar_j - mu_ij - What_ij]; the same iterates, with a
right-hand side that holds only what changed.

Stochastic block subsets (proposed in Sec. 5 and the conclusion, not specified there):
with ``block_fraction`` p < 1, iteration k updates only the blocks drawn active.
Reading: an inactive block (i, j) skips the graph projection and keeps What_ij, O_ij
(and U_ij); every other update, each dual mu_ij included, runs as usual from the
blocks' current values.  The duals of every consensus group then keep summing to zero
(mu_j + sum_i mu_ij = 0 after each averaging step), as in the full method; freezing an
inactive block's mu_ij breaks that sum and the iterates settle at a point whose residuals
vanish but which is not the minimiser.  The draw: block b = i C + j is active in iteration k (from 0) iff
(w >> 8) < floor(p 2^24), w the first word of Philox4x32-10 at counter (b, k, 2, 0)
under the solve's seed (tags 0 and 1 draw G and b); p = 1 keeps every block active.

Stopping: the paper runs a fixed number of iterations; so does this oracle.
Residuals (reported, never used to stop):
  primal = |(O - Obar, W - Wbar, {What_ij - Wbar_j})|_F
  dual   = rho |(Wbar^k - Wbar^{k-1}, Obar^k - Obar^{k-1})|_F

Pins: ridge closed form for squared loss + l2 (Sec. 2.2); the KKT system of the
graph projection; "equation" == "reorganised" == "incremental" to 1e-12; residuals -> 0.
"""
import numpy as np
import scipy.linalg as sla

from . import philox
from . import prox as P
from . import rff


def block_mask(seed, R, C, k, p):
    """Active blocks of iteration k (R x C booleans) for the block fraction p."""
    thr = np.uint64(int(np.floor(float(p) * 2.0 ** 24)))
    k0, k1 = philox.seed_key(seed)
    b = np.arange(R * C, dtype=np.uint64)
    z = np.zeros_like(b)
    w0, _, _, _ = philox.philox4x32_10(b, z + np.uint64(k), z + np.uint64(2), z, k0, k1)
    return ((w0 >> np.uint64(8)) < thr).reshape(R, C)


# ----------------------------------------------------------------- closed forms
def ridge_closed_form(Z, Y, lam):
    """argmin_W |Z W - Y|_F^2 + n lam |W|_F^2 = (Z^T Z + n lam I)^-1 Z^T Y (Sec. 2.2)."""
    Z = np.asarray(Z, dtype=np.float64)
    n, D = Z.shape
    H = Z.T @ Z + n * lam * np.eye(D)
    return sla.solve(H, Z.T @ np.asarray(Y, dtype=np.float64), assume_a="pos")


def graph_projection(A, Xin, Yin, form="auto"):
    """proj_A[(Y, X)] of Sec. 3: argmin 1/2|V - Y|^2 + 1/2|U - X|^2 s.t. V = A U.

    Returns (U, V).  form "gram" uses eq. (graphU): U = (A^T A + I)^-1 (X + A^T Y);
    form "outer" uses the n x n system: U = r - A^T (I + A A^T)^-1 A r with
    r = X + A^T Y (the identity (I + A^T A)^-1 = I - A^T (I + A A^T)^-1 A).
    V = A U (eq. (graphV)).
    """
    A = np.asarray(A, dtype=np.float64)
    n, d = A.shape
    rhs = np.asarray(Xin, dtype=np.float64) + A.T @ np.asarray(Yin, dtype=np.float64)
    if form == "auto":
        form = "gram" if d <= n else "outer"
    if form == "gram":
        U = sla.cho_solve(sla.cho_factor(A.T @ A + np.eye(d), lower=True), rhs)
    elif form == "outer":
        y = sla.cho_solve(sla.cho_factor(A @ A.T + np.eye(n), lower=True), A @ rhs)
        U = rhs - A.T @ y
    else:
        raise ValueError(form)
    return U, A @ U


class _BlockSolver:
    """Cached factor of one block's graph projection (eq. (cache))."""

    def __init__(self, Z):
        self.Z = Z
        n, s = Z.shape
        self.gram = s <= n
        if self.gram:
            self.fac = sla.cho_factor(Z.T @ Z + np.eye(s), lower=True)
        else:
            self.fac = sla.cho_factor(Z @ Z.T + np.eye(n), lower=True)

    def project(self, Xin, Yin):
        Z = self.Z
        rhs = Xin + Z.T @ Yin
        if self.gram:
            U = sla.cho_solve(self.fac, rhs)
        else:
            U = rhs - Z.T @ sla.cho_solve(self.fac, Z @ rhs)
        return U, Z @ U


# ----------------------------------------------------------------- the solver
class Problem:
    """Data and parameters of one solve (Sec. 1, eq. (basicproblem); Sec. 3 grid)."""

    def __init__(self, X, Y, loss="squared", reg="l2", lam=1e-4, sigma=1.0, rho=1.0,
                 D=512, R=1, C=1, seed=0, rho_scale="sum", feature_map="fourier", degree=2, coef0=1.0):
        self.X = np.asarray(X, dtype=np.float64)
        Y = np.asarray(Y, dtype=np.float64)
        self.Y = Y.reshape(Y.shape[0], -1)
        self.n, self.d = self.X.shape
        self.m = self.Y.shape[1]
        if loss not in P.LOSSES or reg not in P.REGS or feature_map not in rff.MAPS:
            raise ValueError("unknown loss/regulariser/feature map")
        if feature_map == "laplace" and (self.X < 0).any():
            raise ValueError("random Laplace features take nonnegative inputs")
        self.feature_map = feature_map
        self.degree, self.coef0 = int(degree), float(coef0)   # TensorSketch: (<x,y>/sigma^2 + coef0)^degree
        self.loss, self.reg = loss, reg
        self.lam, self.sigma, self.rho = float(lam), float(sigma), float(rho)
        self.D, self.R, self.C, self.seed = int(D), int(R), int(C), int(seed)
        if rho_scale == "sum":
            self.t_loss = 1.0 / self.rho
            self.t_reg = self.n * self.lam / self.rho
        elif rho_scale == "mean":
            self.t_loss = 1.0 / (self.n * self.rho)
            self.t_reg = self.lam / self.rho
        else:
            raise ValueError(rho_scale)
        self.rows = rff.partition(self.n, self.R)
        self.cols = rff.partition(self.D, self.C)
        self._Z = None

    def Z(self):
        """The explicit feature matrix, computed once (the oracle stores it)."""
        if self._Z is None:
            self._Z = self._features(self.X)
        return self._Z

    def _features(self, X):
        if self.feature_map == "tensorsketch":   # per-column-block sketches (oracle/tensorsketch.py)
            from . import tensorsketch
            return tensorsketch.features(X, self.seed, self.sigma, self.coef0, self.degree, self.cols)
        return rff.features_block(X, self.seed, self.sigma, self.D, 0, self.D, self.feature_map)

    def solvers(self):
        """Cached factor of every block (eq. (cache)), built on first use."""
        if getattr(self, "_solvers", None) is None:
            self._solvers = [[_BlockSolver(self.Zblock(i, j)) for j in range(self.C)] for i in range(self.R)]
        return self._solvers

    def Zblock(self, i, j):
        r0, r1 = self.rows[i], self.rows[i + 1]
        c0, c1 = self.cols[j], self.cols[j + 1]
        return self.Z()[r0:r1, c0:c1]

    def objective(self, W):
        """sum_i V(y_i, W^T z_i) + n lam r(W)."""
        return P.loss_value(self.loss, self.Y, self.Z() @ W) + self.n * self.lam * P.reg_value(self.reg, W)

    def predict(self, Xq, W):
        """Scores f(x) = W^T z(x) for the rows of Xq."""
        return self._features(np.asarray(Xq, dtype=np.float64)) @ W


def admm(prob, iters, variant="equation", history=False, block_fraction=1.0):
    """Run `iters` iterations; returns a dict of the final state (+ history).

    block_fraction < 1: the stochastic block-subset variant (module header)."""
    R, C, m = prob.R, prob.C, prob.m
    rows, cols = prob.rows, prob.cols
    ni = [int(rows[i + 1] - rows[i]) for i in range(R)]
    sj = [int(cols[j + 1] - cols[j]) for j in range(C)]
    Ys = [prob.Y[rows[i]:rows[i + 1]] for i in range(R)]
    solvers = prob.solvers()

    z = np.zeros
    O = [z((ni[i], m)) for i in range(R)]
    Obar = [z((ni[i], m)) for i in range(R)]
    nu = [z((ni[i], m)) for i in range(R)]
    W = [z((sj[j], m)) for j in range(C)]
    Wbar = [z((sj[j], m)) for j in range(C)]
    mu = [z((sj[j], m)) for j in range(C)]
    What = [[z((sj[j], m)) for j in range(C)] for i in range(R)]
    muij = [[z((sj[j], m)) for j in range(C)] for i in range(R)]
    Obij = [[z((ni[i], m)) for j in range(C)] for i in range(R)]     # equation form
    Oij = [[z((ni[i], m)) for j in range(C)] for i in range(R)]
    U = [[z((sj[j], m)) for j in range(C)] for i in range(R)]        # reorganised
    Dbar = [z((ni[i], m)) for i in range(R)]
    hist = []

    for k in range(iters):
        act = (block_mask(prob.seed, R, C, k, block_fraction) if block_fraction < 1.0
               else np.ones((R, C), dtype=bool))
        Wbar_old = [w.copy() for w in Wbar]
        Obar_old = [o.copy() for o in Obar]
        for i in range(R):
            O[i] = P.prox_loss(prob.loss, Obar[i] - nu[i], Ys[i], prob.t_loss)
        for j in range(C):
            W[j] = P.prox_reg(prob.reg, Wbar[j] - mu[j], prob.t_reg)

        if variant in ("equation", "incremental"):
            for i in range(R):
                for j in range(C):
                    if not act[i, j]:
                        continue
                    if variant == "equation":
                        What[i][j], Oij[i][j] = solvers[i][j].project(Wbar[j] - muij[i][j], Obij[i][j] + nu[i])
                    else:
                        dW, dO = solvers[i][j].project(Wbar[j] - muij[i][j] - What[i][j],
                                                       Obij[i][j] + nu[i] - Oij[i][j])
                        What[i][j], Oij[i][j] = What[i][j] + dW, Oij[i][j] + dO
            for j in range(C):
                Wbar[j] = (W[j] + sum(What[i][j] for i in range(R))) / (R + 1)
            for i in range(R):
                Delta = O[i] - sum(Oij[i][j] for j in range(C))
                for j in range(C):
                    Obij[i][j] = Oij[i][j] + Delta / (C + 1)
                Obar[i] = sum(Obij[i][j] for j in range(C))
            for j in range(C):
                mu[j] = mu[j] + W[j] - Wbar[j]
            for i in range(R):
                for j in range(C):
                    muij[i][j] = muij[i][j] + What[i][j] - Wbar[j]
                nu[i] = nu[i] + O[i] - Obar[i]

        elif variant == "reorganised":
            for i in range(R):
                Zs = [solvers[i][j].Z for j in range(C)]
                corr = Dbar[i] / (C + 1) + nu[i]
                for j in range(C):
                    # Z^T (Obar_ij + nu_i) = U_ij + Z^T (Delta_i/(C+1) + nu_i); the
                    # projection's right-hand side is assembled from these parts
                    # and solved with the cached factor of block (i, j).
                    if not act[i, j]:
                        continue
                    s = solvers[i][j]
                    rhs = Wbar[j] - muij[i][j] + U[i][j] + Zs[j].T @ corr
                    if s.gram:
                        What[i][j] = sla.cho_solve(s.fac, rhs)
                    else:
                        What[i][j] = rhs - Zs[j].T @ sla.cho_solve(s.fac, Zs[j] @ rhs)
                    Oij[i][j] = Zs[j] @ What[i][j]
                    U[i][j] = Zs[j].T @ Oij[i][j]
                S = sum(Oij[i][j] for j in range(C))
                Dbar[i] = O[i] - S
                Obar[i] = S / (C + 1) + (C / (C + 1)) * O[i]
            for j in range(C):
                Wbar[j] = (W[j] + sum(What[i][j] for i in range(R))) / (R + 1)
            for j in range(C):
                mu[j] = mu[j] + W[j] - Wbar[j]
            for i in range(R):
                for j in range(C):
                    muij[i][j] = muij[i][j] + What[i][j] - Wbar[j]
                nu[i] = nu[i] + O[i] - Obar[i]

        elif variant == "algorithm1_literal":
            # Algorithm 1 exactly as printed: no Z^T nu term, and mu', mu
            # updated with the Wbar of the previous iteration.
            if block_fraction < 1.0:
                raise ValueError("the literal Algorithm 1 has no stochastic variant")
            for i in range(R):
                Zs = [solvers[i][j].Z for j in range(C)]
                Delta = O[i].copy()
                Ob = (C / (C + 1)) * O[i]
                for j in range(C):
                    s = solvers[i][j]
                    A = Zs[j].T @ Dbar[i] / (C + 1)
                    rhs = Wbar[j] - muij[i][j] + U[i][j] + A
                    if s.gram:
                        What[i][j] = sla.cho_solve(s.fac, rhs)
                    else:
                        What[i][j] = rhs - Zs[j].T @ sla.cho_solve(s.fac, Zs[j] @ rhs)
                    Op = Zs[j] @ What[i][j]
                    Delta = Delta - Op
                    U[i][j] = Zs[j].T @ Op
                    Ob = Ob + Op / (C + 1)
                    muij[i][j] = muij[i][j] + What[i][j] - Wbar[j]
                Dbar[i] = Delta
                Obar[i] = Ob
            for j in range(C):
                mu[j] = mu[j] + W[j] - Wbar[j]
                Wbar[j] = (sum(What[i][j] for i in range(R)) + W[j]) / (R + 1)
            for i in range(R):
                nu[i] = nu[i] + O[i] - Obar[i]
        else:
            raise ValueError(variant)

        if history:
            pr = sum(np.sum((O[i] - Obar[i]) ** 2) for i in range(R))
            pr += sum(np.sum((W[j] - Wbar[j]) ** 2) for j in range(C))
            pr += sum(np.sum((What[i][j] - Wbar[j]) ** 2) for i in range(R) for j in range(C))
            du = sum(np.sum((Wbar[j] - Wbar_old[j]) ** 2) for j in range(C))
            du += sum(np.sum((Obar[i] - Obar_old[i]) ** 2) for i in range(R))
            hist.append((np.sqrt(pr), prob.rho * np.sqrt(du)))

    cat = np.concatenate
    out = dict(Wbar=cat(Wbar), W=cat(W), mu=cat(mu), O=cat(O), Obar=cat(Obar), nu=cat(nu),
               What=[cat([What[i][j] for j in range(C)]) for i in range(R)],
               muij=[cat([muij[i][j] for j in range(C)]) for i in range(R)],
               Oij=[[Oij[i][j] for j in range(C)] for i in range(R)])
    if history:
        out["history"] = np.array(hist)
    return out
