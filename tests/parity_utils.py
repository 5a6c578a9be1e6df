"""Replay protocol shared by the GPU parity tests and the smoke check.

The oracle runs the closed loop in FP64.  Before every compared cycle its
state is rounded to float32 and loaded into the CUDA context, so that both
sides start the cycle from bit-identical inputs; no value ever flows from the
CUDA path into the oracle.  The plant (Alg. 1, Execute) integrates the
oracle's U_* over one period, and goals drift at their set velocity.
"""
import numpy as np

F32 = np.float32


def r32(x):
    return np.asarray(x, np.float64).astype(F32).astype(np.float64)


def goals(orc, sc):
    gp, gR = [], []
    for a in range(sc.n_arms):
        p, R = orc.goal_pose(a, sc.goal_q[a])
        gp.append(r32(p))
        gR.append(r32(R))
    return np.asarray(gp), np.asarray(gR)


def load_oracle_state(ctl, orc):
    from paper_2602_10114_gb300.mrs import state_blob
    orc.round_state_to_f32()
    s = orc.state
    blob = state_blob(orc.sc, s["mu"], s["Sigma"], orc.cycle_index, orc.world_t, s["plan_valid"],
                      s["plan_stamp"], s["plan_dist"], s["plan_spheres"], s["plan_q"])
    ctl.load_state(blob)


def cost_tol(c_ref):
    """1e-4 relative with an absolute floor of 1e-6 (1 + |C|)."""
    c = np.abs(c_ref)
    return 1e-4 * c + 1e-6 * (1 + c)


class Replay:
    def __init__(self, sc, device="cuda:0", threads=8):
        from oracle.oracle import Oracle
        from paper_2602_10114_gb300 import mrs
        self.sc = sc
        self.orc = Oracle(sc, threads=threads)
        self.ctl = mrs.Controller(sc, device=device)
        self.ctl.set_world()
        self.q = [r32(q) for q in sc.q0]
        self.qd = [r32(q) for q in sc.qd0]
        self.gp, self.gR = goals(self.orc, sc)

    def cycle(self, dump=None):
        load_oracle_state(self.ctl, self.orc)
        got = self.ctl.step([q.astype(F32) for q in self.q], [q.astype(F32) for q in self.qd],
                            self.gp.astype(F32), self.gR.astype(F32))
        got_costs = [self.ctl.debug_costs(a) for a in range(self.sc.n_arms)]
        got_alpha = self.ctl.debug_alpha()
        got_sph = self.ctl.debug_spheres(dump) if dump is not None else None
        exp = self.orc.cycle(self.q, self.qd, self.gp, self.gR, dump=dump, want_U=True)
        return got, got_costs, got_alpha, got_sph, exp

    def advance(self, exp):
        """Plant: integrate the oracle's U_* over one period; drift goals."""
        dt = float(F32(self.sc.params["dt"]))
        for a in range(self.sc.n_arms):
            u = self.orc.split(exp["u_star"], "d", a)
            self.qd[a] = r32(self.qd[a] + u * dt)
            self.q[a] = r32(self.q[a] + self.qd[a] * dt)
            self.gp[a] = r32(self.gp[a] + self.sc.goal_vel[a] * dt)


def parse_state(sc, blob):
    """Inverse of state_blob: (mu, Sigma, cycle, world_t, valid, stamp, dist,
    plan_spheres, plan_q) with per-arm arrays concatenated."""
    import struct
    magic, ver, A, _, cycle, wt, _ = struct.unpack_from("<IIIIqff", blob, 0)
    o = 32
    mu, Sg = [], []
    for a in sc.arms:
        hd, hdd = a.H * a.dof, a.H * a.dof * a.dof
        mu.append(np.frombuffer(blob, np.float32, hd, o)); o += 4 * hd
        Sg.append(np.frombuffer(blob, np.float32, hdd, o)); o += 4 * hdd
    valid, stamp, dist, sph, pq = [], [], [], [], []
    for a in sc.arms:
        v, _, s, d, _ = struct.unpack_from("<iiqff", blob, o); o += 24
        valid.append(v); stamp.append(s); dist.append(d)
        hs, hd = a.H * a.n_spheres * 4, a.H * a.dof
        sph.append(np.frombuffer(blob, np.float32, hs, o)); o += 4 * hs
        pq.append(np.frombuffer(blob, np.float32, hd, o)); o += 4 * hd
    return dict(mu=np.concatenate(mu), Sigma=np.concatenate(Sg), cycle=cycle, world_t=wt,
                valid=np.array(valid), stamp=np.array(stamp), dist=np.array(dist),
                plan_spheres=np.concatenate(sph), plan_q=np.concatenate(pq))


def oracle_weights(costs, lam):
    c = np.asarray(costs, np.float64)
    w = np.exp(-(c - c.min()) / lam)
    return w / w.sum()


# FP32 error model of one clearance distance (m): sphere centres come out of a
# float32 DH chain over about a metre (2^-24 relative rounding per operation,
# a few tens of operations), so a distance is trusted to EPS_D.  The sphere
# parity tests check the observed centre errors against EPS_D / 4.
EPS_D = 2e-6


def cost_error_bound(exp, orc, arm):
    """A priori FP32 error bound of each rollout's total cost: the cost's
    sensitivity to a common distance error (sum of the active ramp slopes,
    reported by the oracle) times EPS_D, plus 1e-6 relative for rounding."""
    c = orc.split(exp["costs"], "k", arm)
    return EPS_D * orc.split(exp["sens"], "k", arm) + 1e-6 * np.abs(c)


def update_tolerance(exp, orc, arm, lam, alpha_mu, alpha_sigma, floor=1e-5):
    """Element-wise tolerance of the updated mean [H][d] and covariance
    [H][d][d]: first-order propagation of the cost error bound through Eqs.
    2-4.  With w_n the weights and e_n the bound of C_n,
      |d mu~_h|    <= (1/lambda) sum_n w_n |U_nh - mu~_h| (e_n + sum_m w_m e_m)
      |d Sigma~_h| <= (1/lambda) sum_n w_n |D_nh - Sigma~_h| (e_n + sum_m w_m e_m)
    with D_nh = (U_nh - mu~_h)(U_nh - mu~_h)^T; the EMA scales them by alpha."""
    c = orc.split(exp["costs"], "k", arm)
    w = oracle_weights(c, lam)
    e = cost_error_bound(exp, orc, arm)
    ee = e + np.dot(w, e)
    U = orc.split(exp["U"], "U", arm)                 # [K][H][d]
    mt = np.einsum("n,nhj->hj", w, U)
    dev = U - mt[None]
    tol_mu = floor + alpha_mu / lam * np.einsum("n,nhj->hj", w * ee, np.abs(dev))
    D = np.einsum("nhj,nhk->nhjk", dev, dev)
    St = np.einsum("n,nhjk->hjk", w, D)
    tol_sig = floor + alpha_sigma / lam * np.einsum("n,nhjk->hjk", w * ee, np.abs(D - St[None]))
    return tol_mu, tol_sig


def fp32_update_bound(exp, orc, arm, lam, alpha_mu, alpha_sigma):
    """Conditioning of one arm's update in FP32, from the oracle alone: the
    first-order change of the updated mean [H][d] and covariance [H][d][d]
    when each total cost C_n carries a realistic FP32 error
      e_n = 2^-22 |C_n| + (EPS_D / 4) S_n
    (four units in the last place of the stored cost, plus the sphere error
    the sphere parity checks enforce, EPS_D / 4, times the cost's ramp
    sensitivity S_n).  To first order in the cost errors dC_n, Eq. 2 moves the
    weights by dw_n = w_n (sum_m w_m dC_m - dC_n) / lambda, and since
    sum_n w_n (U_n - mu~) = 0 the common part cancels in Eq. 3:
      d mu~ = -(1/lambda) sum_n w_n dC_n (U_n - mu~),
    so |d mu~| <= (1/lambda) sum_n w_n e_n |U_n - mu~| (likewise for Sigma~
    with D_n - Sigma~), scaled by the EMA step of Eq. 4.  Where this bound
    exceeds 1e-5 the weights resolve cost differences finer than the FP32
    costs carry: the costs are large against lambda (contact ramps, priority
    weights of up to 1e6 on the coordination term) and several samples keep
    weight, so no FP32 evaluation of the costs can hold the mean to 1e-5."""
    c = orc.split(exp["costs"], "k", arm)
    w = oracle_weights(c, lam)
    e = 2.0 ** -22 * np.abs(c) + EPS_D / 4 * orc.split(exp["sens"], "k", arm)
    U = orc.split(exp["U"], "U", arm)
    mt = np.einsum("n,nhj->hj", w, U)
    dev = U - mt[None]
    b_mu = alpha_mu / lam * np.einsum("n,nhj->hj", w * e, np.abs(dev))
    D = np.einsum("nhj,nhk->nhjk", dev, dev)
    St = np.einsum("n,nhjk->hjk", w, D)
    b_sig = alpha_sigma / lam * np.einsum("n,nhjk->hjk", w * e, np.abs(D - St[None]))
    return float(b_mu.max()), float(b_sig.max())


def plan_tolerance(sc, arm, tol_mu, floor=1e-5, mu_floor=1e-5):
    """Tolerance of the published plan's sphere positions [H]: 1e-5 m plus the
    part of the mean's tolerance above its floor carried through ToPlan.  The
    plan integrates the mean, q_h = q_0 + h dt qd_0 + dt^2 sum_{k<=h} (h-k+1)
    mu_k, and a joint error moves a sphere by at most the arm's reach R times
    that error (R = sum of |a_i| + |d_i| plus 0.2 m for the tool)."""
    a = sc.arms[arm]
    dt = float(np.float32(sc.params["dt"]))
    R = float(np.sum(np.abs(a.dh[:, 0])) + np.sum(np.abs(a.dh[:, 1]))) + 0.2
    ex = np.maximum(tol_mu - mu_floor, 0.0)                      # [H][d]
    H = a.H
    W = np.array([[(h - k + 1) if k <= h else 0 for k in range(H)] for h in range(H)], float)
    dq = dt * dt * (W @ ex)                                      # [H][d]
    return floor + R * dq.sum(axis=1)
