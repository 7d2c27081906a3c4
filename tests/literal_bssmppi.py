"""A literal pure-Python restatement of one BSS-MPPI solve, for brute-force checks on tiny inputs.

Written separately from the C oracle (its own Philox, its own model, its own moments) so that an
indexing or plumbing slip in either one shows up as a disagreement. Everything is Python floats
(IEEE double) and lists; it is only practical for K, M, T of a few units.

Follows Algorithm 1 (sampling, rollout, cost with the augmented belief state, OptimalControl) and
Algorithm 2 (particle propagation, Monte-Carlo mean and unbiased covariance), the trajectory cost
and weights equations, Eq. "cbfpenalty" and Eq. "DCBF".
"""
import math

M32 = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    c = [x & M32 for x in ctr]
    k0, k1 = key[0] & M32, key[1] & M32
    for rnd in range(10):
        if rnd:
            k0 = (k0 + 0x9E3779B9) & M32
            k1 = (k1 + 0xBB67AE85) & M32
        p0 = 0xD2511F53 * c[0]
        p1 = 0xCD9E8D57 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k0) & M32, p1 & M32, ((p0 >> 32) ^ c[3] ^ k1) & M32, p0 & M32]
    return c


def normals(n_out, t, n, k, stream, ctr, seed):
    key = (seed & M32, (seed >> 32) & M32)
    z = []
    words = None
    for i in range((n_out + 1) // 2):
        if i % 2 == 0:
            words = philox4x32_10((t | ((i // 2) << 16), n, k, (stream << 28) | (ctr & 0x0FFFFFFF)), key)
        a, b = words[2 * (i % 2)], words[2 * (i % 2) + 1]
        u1 = ((a >> 8) + 1) / 16777216.0
        u2 = (b >> 8) / 16777216.0
        r = math.sqrt(-2.0 * math.log(u1))
        z += [r * math.cos(2 * math.pi * u2), r * math.sin(2 * math.pi * u2)]
    return z[:n_out]


def disturbance(nx, t, n, k, ctr, seed, M):
    """Disturbance normals of particle n: for 6 states the particles n and n + H (H = half the
    smallest power of two >= M) share a counter keyed by the lower index and split its six pairs."""
    if nx != 6:
        return normals(nx, t, n, k, 1, ctr, seed)
    H = 1
    while 2 * H < M:
        H *= 2
    upper = n >= H
    twelve = normals(12, t, n - H if upper else n, k, 1, ctr, seed)
    return twelve[6:] if upper else twelve[:6]


def chol(A):
    n = len(A)
    L = [[0.0] * n for _ in range(n)]
    for j in range(n):
        d = A[j][j] - sum(L[j][q] ** 2 for q in range(j))
        if d <= 1e-300:
            continue
        L[j][j] = math.sqrt(d)
        for i in range(j + 1, n):
            L[i][j] = (A[i][j] - sum(L[i][q] * L[j][q] for q in range(j))) / L[j][j]
    return L


def kappa_at(P, s):
    n = len(P["kappa"])
    x = s / P["track_len"] * n
    i = math.floor(x)
    f = x - i
    i0 = i % n
    return (1 - f) * P["kappa"][i0] + f * P["kappa"][(i0 + 1) % n]


def f_model(P, x, u):
    if P["model"] == 1:
        dt = P["dt"]
        return [x[0] + dt * x[2] + 0.5 * dt * dt * u[0], x[1] + dt * x[3] + 0.5 * dt * dt * u[1],
                x[2] + dt * u[0], x[3] + dt * u[1]]
    h = P["dt"] / P["n_sub"]
    x = list(x)
    m, lf, lr = P["mass"], P["lf"], P["lr"]
    for _ in range(P["n_sub"]):
        vx, vy, r, ep, ey, s = x
        d, a = u
        vxh = max(vx, P["vx_floor"])
        af = d - math.atan2(vy + lf * r, vxh)
        ar = -math.atan2(vy - lr * r, vxh)
        Ff = P["mu"] * m * P["g"] * lr / (lf + lr) * math.sin(P["tire_C"] * math.atan(P["tire_B"] * af))
        Fr = P["mu"] * m * P["g"] * lf / (lf + lr) * math.sin(P["tire_C"] * math.atan(P["tire_B"] * ar))
        kap = kappa_at(P, s)
        sd = (vx * math.cos(ep) - vy * math.sin(ep)) / (1 - kap * ey)
        dx = [a - Ff * math.sin(d) / m + vy * r, (Ff * math.cos(d) + Fr) / m - vx * r,
              (lf * Ff * math.cos(d) - lr * Fr) / P["Iz"], r - kap * sd,
              vx * math.sin(ep) + vy * math.cos(ep), sd]
        x = [x[i] + h * dx[i] for i in range(6)]
    return x


def solve(P, x0, v, ctr):
    """Returns (S, u, mean, cov, v_plus, w) as nested lists."""
    K, M, T, nx = P["K"], P["M"], P["T"], len(x0)
    e = P["ey_index"]
    Le = chol(P["Sigma_eps"])
    Lw = chol(P["Sigma_w"])
    Se = P["Sigma_eps"]
    det = Se[0][0] * Se[1][1] - Se[0][1] * Se[1][0]
    Si = [[Se[1][1] / det, -Se[0][1] / det], [-Se[1][0] / det, Se[0][0] / det]]
    nu = P["nu"]

    def h_of(mean, cov):
        margin = P["w_T"] - nu * math.sqrt(max(cov[e][e], 0.0))
        if P.get("clamp_margin") and margin < 0.0:
            margin = 0.0
        return margin ** 2 - mean[e] ** 2

    def cost(W, mean):
        c = sum(W[i] * (mean[i] - P["x_goal"][i]) ** 2 for i in range(nx))
        return c + (P["C_obs"] if abs(mean[e]) > P["w_T"] else 0.0)

    def csafe(hn, hp):
        return P["C_safe"] * max(-hn + (1 - P["gamma"]) * hp, 0.0)

    S_all, U_all, MEAN, COV = [], [], [], []
    for m in range(K):
        kk = 0 if P["crn"] else m
        U = []
        for t in range(T):
            z = normals(2, t, 0, m, 0, ctr, P["seed"])
            eps = [Le[0][0] * z[0], Le[1][0] * z[0] + Le[1][1] * z[1]]
            U.append([min(max(v[t][j] + eps[j], P["u_min"][j]), P["u_max"][j]) for j in range(2)])
        X = [list(x0) for _ in range(M)]
        means = [list(x0)]
        covs = [[[0.0] * nx for _ in range(nx)]]
        for t in range(T):
            for n in range(M):
                xn = f_model(P, X[n], U[t])
                z = disturbance(nx, t, n, kk, ctr, P["seed"], M)
                X[n] = [xn[i] + sum(Lw[i][j] * z[j] for j in range(i + 1)) for i in range(nx)]
            mean = [sum(X[n][i] for n in range(M)) / M for i in range(nx)]
            cov = [[sum((X[n][i] - mean[i]) * (X[n][j] - mean[j]) for n in range(M)) / (M - 1)
                    for j in range(nx)] for i in range(nx)]
            means.append(mean)
            covs.append(cov)
        hs = [h_of(means[t], covs[t]) for t in range(T + 1)]
        S = 0.0
        for t in range(T):
            ctrl = sum(v[t][i] * Si[i][j] * U[t][j] for i in range(2) for j in range(2))
            S += cost(P["Q"], means[t]) + P["ctrl_w"] * ctrl + csafe(hs[t], hs[t - 1] if t else hs[0])
        S += cost(P["Qf"], means[T]) + csafe(hs[T], hs[T - 1])
        S_all.append(S)
        U_all.append(U)
        MEAN.append(means)
        COV.append(covs)
    beta = min(S_all)
    om = [math.exp(-(s - beta) / P["lam"]) for s in S_all]
    eta = sum(om)
    vp = [[sum(om[m] * U_all[m][t][j] for m in range(K)) / eta for j in range(2)] for t in range(T)]
    return S_all, U_all, MEAN, COV, vp, [o / eta for o in om]


def problem_dict(prob, nu):
    """Plain-dict view of a workload.Problem with float32-rounded constants (as the oracle takes them)."""
    import numpy as np
    f = lambda x: float(np.float32(x))
    nx = prob.nx
    return dict(
        K=prob.K, M=prob.M, T=prob.T, n_sub=prob.n_sub, model=prob.model, dt=f(prob.dt), mass=f(prob.mass),
        Iz=f(prob.Iz), lf=f(prob.lf), lr=f(prob.lr), tire_B=f(prob.tire_B), tire_C=f(prob.tire_C),
        mu=f(prob.mu), g=f(prob.g), vx_floor=f(prob.vx_floor), u_min=[f(x) for x in prob.u_min],
        u_max=[f(x) for x in prob.u_max], Sigma_eps=np.asarray(prob.Sigma_eps, float).tolist(),
        Sigma_w=np.asarray(prob.Sigma_w, float).reshape(nx, nx).tolist(), lam=f(prob.lam),
        gamma=f(prob.gamma), ctrl_w=f(prob.ctrl_w), C_safe=f(prob.C_safe), C_obs=f(prob.C_obs),
        w_T=f(prob.w_T), x_goal=[f(x) for x in prob.x_goal], Q=[f(x) for x in prob.Q],
        Qf=[f(x) for x in prob.Qf], ey_index=prob.ey_index, kappa=[float(k) for k in prob.kappa],
        track_len=f(prob.track_len), seed=int(prob.seed), crn=int(prob.crn_disturbance), nu=nu,
        clamp_margin=int(getattr(prob, "clamp_margin", 0)))
