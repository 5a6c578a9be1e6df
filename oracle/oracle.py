"""ctypes front end of the FP64 CPU oracle (mrs_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg use it; the library path never does.  It marshals a
`Scenario` (float32 inputs) into double arrays, owns the controller state,
and exposes the oracle's functions one by one for the pins.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmrs_oracle.so")
SRC = os.path.join(HERE, "mrs_oracle.c")

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_llp = C.POINTER(C.c_longlong)


class OrcArm(C.Structure):
    _fields_ = [("dof", C.c_int), ("n_spheres", C.c_int), ("K", C.c_int), ("H", C.c_int),
                ("dh", _dp), ("q_lo", _dp), ("q_hi", _dp), ("qd_max", _dp),
                ("sphere_body", _ip), ("sphere_xyzr", _dp), ("base_pose", C.c_double * 7)]


class OrcConfig(C.Structure):
    _fields_ = [("n_arms", C.c_int), ("arms", C.POINTER(OrcArm)),
                ("dt", C.c_double), ("lambda_", C.c_double), ("gamma", C.c_double),
                ("alpha_mu", C.c_double), ("alpha_sigma", C.c_double),
                ("sigma_init", C.c_double), ("w_pose", C.c_double), ("w_rot", C.c_double),
                ("w_stop", C.c_double), ("w_joint", C.c_double), ("w_coll", C.c_double),
                ("w_self", C.c_double), ("w_dyn", C.c_double), ("B", C.c_double),
                ("B_world", C.c_double), ("B_self", C.c_double), ("tau", C.c_double),
                ("q_margin", C.c_double), ("iterations", C.c_int), ("seed", C.c_uint64),
                ("max_plan_age", C.c_int), ("active", _ip), ("w_manip", C.c_double),
                ("manip_w0", C.c_double)]


class OrcState(C.Structure):
    _fields_ = [("mu", _dp), ("Sigma", _dp), ("cycle", C.c_longlong), ("world_t", C.c_double),
                ("plan_valid", _ip), ("plan_stamp", _llp), ("plan_dist", _dp),
                ("plan_spheres", _dp), ("plan_q", _dp)]


class OrcInputs(C.Structure):
    _fields_ = [("q", _dp), ("qd", _dp), ("goal_p", _dp), ("goal_R", _dp),
                ("n_world", C.c_int), ("world", _dp), ("world_vel", _dp),
                ("n_aabb", C.c_int), ("aabb", _dp)]


class OrcOutputs(C.Structure):
    _fields_ = [("mean_plan", _dp), ("Sigma", _dp), ("plan_spheres", _dp), ("plan_q", _dp),
                ("u_star", _dp), ("dist_to_goal", _dp), ("min_cost", _dp), ("n_star", _ip),
                ("costs", _dp), ("alpha", _dp), ("n_queries", _llp), ("sens", _dp),
                ("U", _dp), ("n_dump", C.c_int),
                ("dump_anh", _ip), ("dump_spheres", _dp), ("dump_stage", _dp)]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               SRC, "-o", LIB_PATH, "-lm"]
        subprocess.check_call(cmd)
    return LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB_PATH)
            L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
            L.orc_uniform23.restype = C.c_double
            L.orc_uniform23.argtypes = [C.c_uint32]
            L.orc_normals.argtypes = [C.c_uint64, C.c_int, C.c_longlong, C.c_int, C.c_int,
                                      C.c_int, C.c_int, _dp]
            L.orc_cholesky.argtypes = [C.c_int, _dp, C.c_double, _dp]
            L.orc_fk.argtypes = [C.POINTER(OrcArm), _dp, _dp, _dp]
            L.orc_sphere_sphere.restype = C.c_double
            L.orc_sphere_sphere.argtypes = [_dp, _dp]
            L.orc_sphere_aabb.restype = C.c_double
            L.orc_sphere_aabb.argtypes = [_dp, _dp]
            L.orc_pose_cost.restype = C.c_double
            L.orc_pose_cost.argtypes = [_dp, _dp, _dp, C.c_double]
            L.orc_stop_cost.restype = C.c_double
            L.orc_stop_cost.argtypes = [C.c_int, _dp, _dp]
            L.orc_joint_cost.restype = C.c_double
            L.orc_joint_cost.argtypes = [C.c_int, _dp, _dp, _dp, C.c_double]
            L.orc_ramp.restype = C.c_double
            L.orc_ramp.argtypes = [C.c_double, C.c_double]
            L.orc_priority.restype = C.c_double
            L.orc_priority.argtypes = [C.c_double, C.c_double, C.c_double]
            L.orc_weights.argtypes = [C.c_int, _dp, C.c_double, _dp]
            L.orc_query_count.restype = C.c_longlong
            L.orc_query_count.argtypes = [C.POINTER(OrcConfig), C.c_int]
            L.orc_init_state.argtypes = [C.POINTER(OrcConfig), C.POINTER(OrcState)]
            L.orc_cycle.restype = C.c_int
            L.orc_cycle.argtypes = [C.POINTER(OrcConfig), C.POINTER(OrcState),
                                    C.POINTER(OrcInputs), C.POINTER(OrcOutputs)]
            L.orc_rollout.restype = C.c_double
            L.orc_rollout.argtypes = [C.POINTER(OrcConfig), C.c_int, C.POINTER(OrcState),
                                      C.POINTER(OrcInputs), _dp, _dp, _dp, _dp, _dp, _llp, _dp]
            L.orc_sample_costs.restype = C.c_int
            L.orc_sample_costs.argtypes = [C.POINTER(OrcConfig), C.POINTER(OrcState),
                                           C.POINTER(OrcInputs), C.c_int, C.c_int, _ip, _dp, _dp]
            L.orc_mlp_loss_grad.restype = C.c_double
            L.orc_mlp_loss_grad_w.restype = C.c_double
            L.orc_mlp_loss_grad_w.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _dp, C.c_int, _dp,
                                              _dp, C.c_double, _dp, _dp]
            L.orc_mlp_loss_grad.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _dp, C.c_int, _dp,
                                            _dp, _dp, _dp]
            L.orc_self_distance.argtypes = [C.POINTER(OrcArm), C.c_int, _dp, C.c_double, _dp]
            L.orc_self_pair_used.restype = C.c_int
            L.orc_self_pair_used.argtypes = [C.POINTER(OrcArm), C.c_int, C.c_int, C.c_double]
            L.orc_jacobian.argtypes = [C.POINTER(OrcArm), _dp, _dp]
            L.orc_manipulability.restype = C.c_double
            L.orc_manipulability.argtypes = [C.c_int, _dp]
            L.orc_manip_cost.restype = C.c_double
            L.orc_manip_cost.argtypes = [C.c_double, C.c_double]
            L.orc_pair_distance.argtypes = [C.POINTER(OrcArm), C.POINTER(OrcArm), C.c_int, _dp,
                                            _dp, _dp]
            L.orc_pair_distance_posed.argtypes = [C.POINTER(OrcArm), C.POINTER(OrcArm), C.c_int,
                                                  _dp, _dp, _dp, _dp]
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_get_threads.restype = C.c_int
            _lib = L
    return _lib


def _d(a):
    """Contiguous float64 copy (kept alive by the caller) and its pointer."""
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return arr, arr.ctypes.data_as(_dp)


def _ptr(arr, t=_dp):
    return None if arr is None else arr.ctypes.data_as(t)


# ---------------------------------------------------------------------------
# single functions, for the pins

def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xffffffff for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xffffffff for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def uniform23(x):
    return lib().orc_uniform23(int(x) & 0xffffffff)


def normals(seed, arm, cycle, it, n, h, d):
    z = np.zeros(d)
    lib().orc_normals(seed, arm, cycle, it, n, h, d, _ptr(z))
    return z


def cholesky(S, jitter=1e-8):
    S = np.ascontiguousarray(S, dtype=np.float64)
    d = S.shape[0]
    L = np.zeros((d, d))
    lib().orc_cholesky(d, _ptr(S), jitter, _ptr(L))
    return L


def sphere_sphere(a, b):
    a, pa = _d(a)
    b, pb = _d(b)
    return lib().orc_sphere_sphere(pa, pb)


def sphere_aabb(s, box):
    s, ps = _d(s)
    b, pb = _d(box)
    return lib().orc_sphere_aabb(ps, pb)


def pose_cost(T, goal_p, goal_R, w_rot):
    T, pT = _d(T)
    g, pg = _d(goal_p)
    R, pR = _d(goal_R)
    return lib().orc_pose_cost(pT, pg, pR, w_rot)


def stop_cost(qd, qd_max):
    qd, p1 = _d(qd)
    m, p2 = _d(qd_max)
    return lib().orc_stop_cost(len(qd), p1, p2)


def joint_cost(q, lo, hi, margin):
    q, p1 = _d(q)
    lo, p2 = _d(lo)
    hi, p3 = _d(hi)
    return lib().orc_joint_cost(len(q), p1, p2, p3, margin)


def ramp(dist, B):
    return lib().orc_ramp(dist, B)


def priority(e_self, e_other, tau):
    return lib().orc_priority(e_self, e_other, tau)


def weights(Cn, lam):
    Cn, p = _d(Cn)
    w = np.zeros(len(Cn))
    lib().orc_weights(len(Cn), p, lam, _ptr(w))
    return w


def manip_cost(w, w0):
    return float(lib().orc_manip_cost(float(w), float(w0)))


def mlp_loss_grad(in_dim, width, layers, params, x, t, want_grad=True, over_weight=1.0):
    """FP64 loss, gradient and outputs of the surrogate MLP (over-predictions
    weighted by over_weight)."""
    in_pad = (in_dim + 15) // 16 * 16
    p, pp = _d(params)
    x, px = _d(x)
    t, pt = _d(t)
    g = np.zeros(len(p)) if want_grad else None
    y = np.zeros(len(t))
    loss = lib().orc_mlp_loss_grad_w(in_dim, in_pad, width, layers, pp, len(t), px, pt,
                                     float(over_weight), _ptr(g), _ptr(y))
    return loss, g, y


# ---------------------------------------------------------------------------
# whole-scenario front end

class Oracle:
    """Owns the marshalled arms/config and the controller state of one
    scenario; `cycle()` runs Algorithm 1 once for every arm."""

    def __init__(self, sc, threads: int = 1, active=None):
        self.sc = sc
        L = lib()
        L.orc_set_threads(int(threads))
        self._keep = []
        A = sc.n_arms
        self.arms = (OrcArm * A)()
        for i, a in enumerate(sc.arms):
            dh, pdh = _d(a.dh)
            lo, plo = _d(a.q_lo)
            hi, phi = _d(a.q_hi)
            vm, pvm = _d(a.qd_max)
            body = np.ascontiguousarray(a.sphere_body, dtype=np.int32)
            xyzr, pxyzr = _d(a.sphere_xyzr)
            self._keep += [dh, lo, hi, vm, body, xyzr]
            s = self.arms[i]
            s.dof, s.n_spheres, s.K, s.H = a.dof, a.n_spheres, a.K, a.H
            s.dh, s.q_lo, s.q_hi, s.qd_max = pdh, plo, phi, pvm
            s.sphere_body = body.ctypes.data_as(_ip)
            s.sphere_xyzr = pxyzr
            for k in range(7):
                s.base_pose[k] = float(a.base_pose[k])
        # the CUDA path reads float32 parameters: use exactly those values
        p = {k: (v if k in ("iterations", "seed") else float(np.float32(v)))
             for k, v in sc.params.items()}
        self.cfg = OrcConfig(A, self.arms, p["dt"], p["lam"], p["gamma"], p["alpha_mu"],
                             p["alpha_sigma"], p["sigma_init"], p["w_pose"], p["w_rot"],
                             p["w_stop"], p["w_joint"], p["w_coll"], p["w_self"], p["w_dyn"],
                             p["B"], p["B_world"], p["B_self"], p["tau"], p["q_margin"],
                             int(p["iterations"]), int(p["seed"]), int(p.get("max_plan_age", 0)),
                             None, p.get("w_manip", 0.0), p.get("manip_w0", 0.02))
        if active is not None:          # arms this controller optimises
            self._active = np.ascontiguousarray(active, dtype=np.int32)
            self.cfg.active = self._active.ctypes.data_as(_ip)
        self.hd = [a.H * a.dof for a in sc.arms]
        self.hdd = [a.H * a.dof * a.dof for a in sc.arms]
        self.hs = [a.H * a.n_spheres * 4 for a in sc.arms]
        self.off_hd = np.concatenate([[0], np.cumsum(self.hd)]).astype(int)
        self.off_hdd = np.concatenate([[0], np.cumsum(self.hdd)]).astype(int)
        self.off_hs = np.concatenate([[0], np.cumsum(self.hs)]).astype(int)
        self.off_d = np.concatenate([[0], np.cumsum([a.dof for a in sc.arms])]).astype(int)
        self.off_k = np.concatenate([[0], np.cumsum([a.K for a in sc.arms])]).astype(int)
        self.state = dict(
            mu=np.zeros(self.off_hd[-1]), Sigma=np.zeros(self.off_hdd[-1]),
            plan_valid=np.zeros(A, np.int32), plan_stamp=np.zeros(A, np.int64),
            plan_dist=np.zeros(A), plan_spheres=np.zeros(self.off_hs[-1]),
            plan_q=np.zeros(self.off_hd[-1]))
        self.cycle_index = 0
        self.world_t = 0.0
        st = self._state_struct()
        L.orc_init_state(C.byref(self.cfg), C.byref(st))
        self._pull(st)

    # -- state marshalling --------------------------------------------------
    def _state_struct(self):
        s = self.state
        return OrcState(_ptr(s["mu"]), _ptr(s["Sigma"]), self.cycle_index, self.world_t,
                        _ptr(s["plan_valid"], _ip), _ptr(s["plan_stamp"], _llp),
                        _ptr(s["plan_dist"]), _ptr(s["plan_spheres"]), _ptr(s["plan_q"]))

    def _pull(self, st):
        self.cycle_index = int(st.cycle)
        self.world_t = float(st.world_t)

    def round_state_to_f32(self):
        """Round every floating state entry to float32, so that a float32
        consumer can be loaded with exactly the state this oracle continues from."""
        for k in ("mu", "Sigma", "plan_dist", "plan_spheres", "plan_q"):
            self.state[k][:] = self.state[k].astype(np.float32).astype(np.float64)
        self.world_t = float(np.float32(self.world_t))

    def set_world_time(self, t: float):
        self.world_t = float(t)

    # -- inputs -------------------------------------------------------------
    def inputs(self, q, qd, goal_p, goal_R):
        sc = self.sc
        keep = []

        def arr(x):
            a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
            keep.append(a)
            return a.ctypes.data_as(_dp)

        w = np.asarray(sc.world, np.float64).reshape(-1, 4)
        vel = None if sc.world_vel is None else arr(sc.world_vel)
        aabb = np.asarray(sc.aabb, np.float64).reshape(-1, 6)
        inp = OrcInputs(arr(np.concatenate(q)), arr(np.concatenate(qd)), arr(goal_p),
                        arr(goal_R), len(w), arr(w) if len(w) else None, vel,
                        len(aabb), arr(aabb) if len(aabb) else None)
        return inp, keep

    # -- kinematics ---------------------------------------------------------
    def fk(self, arm: int, q):
        a = self.sc.arms[arm]
        q, pq = _d(q)
        frames = np.zeros((a.dof + 1, 4, 4))
        sph = np.zeros((a.n_spheres, 4))
        lib().orc_fk(C.byref(self.arms[arm]), pq, _ptr(frames), _ptr(sph))
        return frames, sph

    def self_distance(self, arm: int, q):
        """Exact self-collision clearance of joint vectors q [n][dof] over the
        arm's self-collision pair set (rest-pose band B_self)."""
        q, pq = _d(np.asarray(q, np.float64).reshape(-1, self.sc.arms[arm].dof))
        out = np.zeros(len(q))
        lib().orc_self_distance(C.byref(self.arms[arm]), len(q), pq, self.cfg.B_self, _ptr(out))
        return out

    def self_pairs(self, arm: int):
        """The arm's self-collision pair set as (s1, s2) index pairs, s1 < s2."""
        n = self.sc.arms[arm].n_spheres
        f = lib().orc_self_pair_used
        return [(i, j) for i in range(n) for j in range(i + 1, n)
                if f(C.byref(self.arms[arm]), i, j, self.cfg.B_self)]

    def pair_distance(self, a: int, b: int, qa, qb, base_b=None, base_a=None):
        """Exact clearance between arm a at joints qa [n][d_a] and arm b at qb
        [n][d_b], each at its base pose (replaced by `base_a` / `base_b`, xyz +
        quaternion w x y z, when given)."""
        qa, pqa = _d(np.asarray(qa, np.float64).reshape(-1, self.sc.arms[a].dof))
        qb, pqb = _d(np.asarray(qb, np.float64).reshape(-1, self.sc.arms[b].dof))
        assert len(qa) == len(qb)
        def with_base(i, base):
            arm = self.arms[i]
            if base is not None:
                arm = OrcArm.from_buffer_copy(self.arms[i])
                for k in range(7):
                    arm.base_pose[k] = float(base[k])
            return arm
        arm_a, arm_b = with_base(a, base_a), with_base(b, base_b)
        out = np.zeros(len(qa))
        lib().orc_pair_distance(C.byref(arm_a), C.byref(arm_b), len(qa), pqa, pqb, _ptr(out))
        return out

    def pair_distance_posed(self, a: int, b: int, qa, qb, pose_b):
        """Clearance of arm a (at its own base frame) at joints qa [n][d_a] and
        arm b at joints qb [n][d_b] placed at pose_b [n][7] in a's frame."""
        qa, pqa = _d(np.asarray(qa, np.float64).reshape(-1, self.sc.arms[a].dof))
        qb, pqb = _d(np.asarray(qb, np.float64).reshape(-1, self.sc.arms[b].dof))
        po, ppo = _d(np.asarray(pose_b, np.float64).reshape(-1, 7))
        assert len(qa) == len(qb) == len(po)
        out = np.zeros(len(qa))
        lib().orc_pair_distance_posed(C.byref(self.arms[a]), C.byref(self.arms[b]), len(qa), pqa,
                                      pqb, ppo, _ptr(out))
        return out

    def jacobian(self, arm: int, q):
        """End-effector geometric Jacobian [6][dof] at joints q."""
        frames, _ = self.fk(arm, q)
        d = self.sc.arms[arm].dof
        f, pf = _d(frames)
        J = np.zeros((6, d))
        lib().orc_jacobian(C.byref(self.arms[arm]), pf, _ptr(J))
        return J

    def manipulability(self, arm: int, q):
        J = self.jacobian(arm, q)
        j, pj = _d(J)
        return float(lib().orc_manipulability(self.sc.arms[arm].dof, pj))

    def goal_pose(self, arm: int, q):
        frames, _ = self.fk(arm, q)
        T = frames[-1]
        return T[:3, 3].copy(), T[:3, :3].copy()

    def query_count(self, arm: int) -> int:
        return int(lib().orc_query_count(C.byref(self.cfg), arm))

    # -- one control cycle --------------------------------------------------
    def cycle(self, q, qd, goal_p, goal_R, dump=None, want_costs=True, want_U=False):
        sc = self.sc
        A = sc.n_arms
        inp, keep = self.inputs(q, qd, goal_p, goal_R)
        nsmax = max(a.n_spheres for a in sc.arms)
        out = dict(mean_plan=np.zeros(self.off_hd[-1]), Sigma=np.zeros(self.off_hdd[-1]),
                   plan_spheres=np.zeros(self.off_hs[-1]), plan_q=np.zeros(self.off_hd[-1]),
                   u_star=np.zeros(self.off_d[-1]), dist_to_goal=np.zeros(A),
                   min_cost=np.zeros(A), n_star=np.zeros(A, np.int32),
                   costs=np.zeros(self.off_k[-1]) if want_costs else None,
                   alpha=np.zeros(A * A), n_queries=np.zeros(A, np.int64),
                   sens=np.zeros(self.off_k[-1]) if want_costs else None,
                   U=np.zeros(sum(a.K * a.H * a.dof for a in sc.arms)) if want_U else None)
        dump = np.zeros((0, 3), np.int32) if dump is None else np.ascontiguousarray(dump, np.int32)
        out["dump_spheres"] = np.zeros((len(dump), nsmax, 4))
        out["dump_stage"] = np.zeros(len(dump))
        o = OrcOutputs(_ptr(out["mean_plan"]), _ptr(out["Sigma"]), _ptr(out["plan_spheres"]),
                       _ptr(out["plan_q"]), _ptr(out["u_star"]), _ptr(out["dist_to_goal"]),
                       _ptr(out["min_cost"]), _ptr(out["n_star"], _ip), _ptr(out["costs"]),
                       _ptr(out["alpha"]), _ptr(out["n_queries"], _llp), _ptr(out["sens"]),
                       _ptr(out["U"]), len(dump),
                       _ptr(dump, _ip), _ptr(out["dump_spheres"]), _ptr(out["dump_stage"]))
        st = self._state_struct()
        rc = lib().orc_cycle(C.byref(self.cfg), C.byref(st), C.byref(inp), C.byref(o))
        if rc != 0:
            raise RuntimeError("oracle cycle failed")
        self._pull(st)
        return out

    def rollout(self, arm, q, qd, goal_p, goal_R, U, alpha_row=None):
        """One control sequence U [H][d] of `arm` through f: returns
        (total cost, stage costs [H], spheres [H][NS][4], q [H][d])."""
        a = self.sc.arms[arm]
        inp, keep = self.inputs(q, qd, goal_p, goal_R)
        U, pU = _d(U)
        alpha_row = np.zeros(self.sc.n_arms) if alpha_row is None else alpha_row
        al, pal = _d(alpha_row)
        stage = np.zeros(a.H)
        sph = np.zeros((a.H, a.n_spheres, 4))
        qo = np.zeros((a.H, a.dof))
        nq = C.c_longlong(0)
        sens = C.c_double(0)
        st = self._state_struct()
        tot = lib().orc_rollout(C.byref(self.cfg), arm, C.byref(st), C.byref(inp), pal, pU,
                                _ptr(stage), _ptr(sph), _ptr(qo), C.byref(nq), C.byref(sens))
        self.last_rollout_sens = sens.value
        return tot, stage, sph, qo

    def sample_costs(self, arm, q, qd, goal_p, goal_R, ns, want_spheres=False):
        """Costs of samples `ns` of the next cycle's first iteration, one by
        one (the state is not modified); optionally their sphere trajectories."""
        a = self.sc.arms[arm]
        inp, keep = self.inputs(q, qd, goal_p, goal_R)
        ns = np.ascontiguousarray(ns, dtype=np.int32)
        costs = np.zeros(len(ns))
        sph = np.zeros((len(ns), a.H, a.n_spheres, 4)) if want_spheres else None
        st = self._state_struct()
        rc = lib().orc_sample_costs(C.byref(self.cfg), C.byref(st), C.byref(inp), arm, len(ns),
                                    _ptr(ns, _ip), _ptr(costs), _ptr(sph))
        if rc != 0:
            raise RuntimeError("oracle sample_costs failed")
        return (costs, sph) if want_spheres else costs

    def split(self, flat, kind: str, arm: int):
        """Per-arm view of a concatenated state/output array."""
        a = self.sc.arms[arm]
        if kind == "hd":
            return flat[self.off_hd[arm]:self.off_hd[arm + 1]].reshape(a.H, a.dof)
        if kind == "hdd":
            return flat[self.off_hdd[arm]:self.off_hdd[arm + 1]].reshape(a.H, a.dof, a.dof)
        if kind == "hs":
            return flat[self.off_hs[arm]:self.off_hs[arm + 1]].reshape(a.H, a.n_spheres, 4)
        if kind == "d":
            return flat[self.off_d[arm]:self.off_d[arm + 1]]
        if kind == "k":
            return flat[self.off_k[arm]:self.off_k[arm + 1]]
        if kind == "U":
            o = sum(b.K * b.H * b.dof for b in self.sc.arms[:arm])
            return flat[o:o + a.K * a.H * a.dof].reshape(a.K, a.H, a.dof)
        raise KeyError(kind)
