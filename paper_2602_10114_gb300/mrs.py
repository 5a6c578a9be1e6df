"""Python binding of libmrs (include/mrs.h): argument marshalling only.

Every step of the control cycle runs in the library's CUDA kernels; this
module converts numpy / torch arguments to the C ABI and back.  PyTorch
supplies device memory (the workspace) and streams.  If the compiled library
is missing, loading fails with an error: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int)

STATUS = {0: "MRS_OK", 1: "MRS_EINVAL", 2: "MRS_ENOMEM", 3: "MRS_ECUDA", 4: "MRS_ETIMEOUT",
          5: "MRS_ESTATE", 6: "MRS_EUNSUPPORTED"}

MAX_SPHERES = 64


class MrsArmDesc(C.Structure):
    _fields_ = [("dof", C.c_int), ("n_spheres", C.c_int), ("K", C.c_int), ("H", C.c_int),
                ("dh", _fp), ("q_lo", _fp), ("q_hi", _fp), ("qd_max", _fp),
                ("sphere_body", _ip), ("sphere_xyzr", _fp), ("base_pose", C.c_float * 7),
                ("external", C.c_int)]


class MrsConfig(C.Structure):
    _fields_ = [("n_arms", C.c_int), ("arms", C.POINTER(MrsArmDesc)),
                ("dt", C.c_float), ("lambda_", C.c_float), ("gamma", C.c_float),
                ("alpha_mu", C.c_float), ("alpha_sigma", C.c_float), ("sigma_init", C.c_float),
                ("w_pose", C.c_float), ("w_rot", C.c_float), ("w_stop", C.c_float),
                ("w_joint", C.c_float), ("w_coll", C.c_float), ("w_self", C.c_float),
                ("w_dyn", C.c_float), ("B", C.c_float), ("B_world", C.c_float),
                ("B_self", C.c_float), ("tau", C.c_float), ("q_margin", C.c_float),
                ("iterations", C.c_int), ("seed", C.c_ulonglong), ("reserved", C.c_int),
                ("max_plan_age", C.c_int), ("w_manip", C.c_float), ("manip_w0", C.c_float)]


class MrsArmState(C.Structure):
    _fields_ = [("q", _fp), ("qd", _fp), ("goal_p", _fp), ("goal_R", _fp)]


class MrsStepOut(C.Structure):
    _fields_ = [("mean_plan", _fp), ("plan_spheres", _fp), ("plan_q", _fp), ("u_star", _fp),
                ("dist_to_goal", _fp), ("min_cost", _fp)]


class MrsRolloutShape(C.Structure):
    _fields_ = [("tile_samples", C.c_int), ("blocks_per_sm", C.c_int), ("order", C.c_int),
                ("cycle_ms", C.c_float)]


class MrsSizes(C.Structure):
    _fields_ = [("n_arms", C.c_size_t), ("hd", C.c_size_t), ("hs", C.c_size_t),
                ("d", C.c_size_t), ("k", C.c_size_t), ("hdd", C.c_size_t),
                ("input_floats", C.c_size_t), ("output_floats", C.c_size_t),
                ("state_bytes", C.c_size_t), ("workspace_bytes", C.c_size_t)]


# exported symbol -> (restype, argtypes)
SIGNATURES = {
    "mrs_create": (C.c_int, [C.POINTER(MrsConfig), C.c_void_p, C.POINTER(C.c_void_p)]),
    "mrs_destroy": (None, [C.c_void_p]),
    "mrs_last_error": (C.c_char_p, [C.c_void_p]),
    "mrs_query_sizes": (C.c_int, [C.c_void_p, C.POINTER(MrsSizes)]),
    "mrs_workspace_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "mrs_bind_workspace": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "mrs_set_world": (C.c_int, [C.c_void_p, _fp, _fp, C.c_int, _fp, C.c_int]),
    "mrs_share_plans": (C.c_int, [C.c_void_p, C.c_int, _fp, _fp, C.c_float, C.c_longlong]),
    "mrs_step": (C.c_int, [C.c_void_p, C.POINTER(MrsArmState), C.POINTER(MrsStepOut)]),
    "mrs_step_device": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mrs_output_device": (C.c_int, [C.c_void_p, C.POINTER(MrsStepOut)]),
    "mrs_output_host": (C.c_int, [C.c_void_p, C.POINTER(MrsStepOut)]),
    "mrs_sync": (C.c_int, [C.c_void_p, C.c_double]),
    "mrs_use_graph": (C.c_int, [C.c_void_p, C.c_int]),
    "mrs_save_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "mrs_load_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "mrs_fk": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _fp, _fp, _fp]),
    "mrs_fk_static": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _fp, _fp, _fp]),
    "mrs_debug_costs": (C.c_int, [C.c_void_p, C.c_int, _fp]),
    "mrs_debug_spheres": (C.c_int, [C.c_void_p, C.c_int, _ip, _fp]),
    "mrs_debug_alpha": (C.c_int, [C.c_void_p, _fp]),
    "mrs_set_zero_noise": (C.c_int, [C.c_void_p, C.c_int]),
    "mrs_set_wait_limit": (C.c_int, [C.c_void_p, C.c_longlong]),
    "mrs_enable_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "mrs_kernel_times": (C.c_int, [C.c_void_p, _fp, C.POINTER(C.c_int)]),
    "mrs_set_rollout_shape": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mrs_get_rollout_shape": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]),
    "mrs_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_int),
                               C.c_void_p]),
    "mrs_philox": (C.c_int, [C.c_int, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                             C.POINTER(C.c_uint32)]),
    "mrs_mlp_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_ulonglong, C.c_void_p,
                                 C.POINTER(C.c_void_p)]),
    "mrs_mlp_destroy": (None, [C.c_void_p]),
    "mrs_mlp_last_error": (C.c_char_p, [C.c_void_p]),
    "mrs_mlp_param_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "mrs_mlp_launch_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_int]),
    "mrs_mlp_set_loss": (C.c_int, [C.c_void_p, C.c_float]),
    "mrs_set_pair_surrogate": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_float]),
    "mrs_relative_pose": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _fp]),
    "mrs_pair_dataset": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_ulonglong, _fp,
                                   C.c_int, C.c_float, C.c_float, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p]),
    "mrs_debug_pair": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _fp, _fp]),
    "mrs_mlp_get_params": (C.c_int, [C.c_void_p, _fp, C.c_size_t]),
    "mrs_mlp_set_params": (C.c_int, [C.c_void_p, _fp, C.c_size_t]),
    "mrs_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "mrs_mlp_grads": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, _fp, _fp]),
    "mrs_mlp_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_float, _fp]),
    "mrs_set_self_surrogate": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_float]),
    "mrs_self_dataset": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_ulonglong, C.c_void_p,
                                   C.c_void_p, C.c_void_p]),
    "mrs_self_distance": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "mrs_debug_self": (C.c_int, [C.c_void_p, C.c_int, _fp, _fp]),
    "mrs_selftest_gemm": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_uint16),
                                    C.POINTER(C.c_uint16), _fp]),
}

_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = False):
    """Load libmrs.so from the source tree (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libmrs.so is not built ({path}); run __graft_entry__.build()")
        _build.build()
    L = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class MrsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _pf(a):
    return None if a is None else a.ctypes.data_as(_fp)


def philox(ctr, key):
    """Device Philox4x32-10 of counters ctr [n][4] under key [2] -> [n][4]."""
    L = load()
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.zeros_like(ctr)
    p = C.POINTER(C.c_uint32)
    st = L.mrs_philox(len(ctr), ctr.ctypes.data_as(p), key.ctypes.data_as(p), out.ctypes.data_as(p))
    if st != 0:
        raise MrsError(st, "philox self-test")
    return out


class Controller:
    """One library context for a `scenarios.Scenario` (or any object with the
    same fields).  The device workspace is a torch uint8 tensor on `device`."""

    def __init__(self, sc, device="cuda", stream=None, workspace=True, external=()):
        import torch
        self.L = load()
        self.sc = sc
        self._keep = []
        A = len(sc.arms)
        self._arms = (MrsArmDesc * A)()
        for i, a in enumerate(sc.arms):
            dh, lo, hi, vm = _f32(a.dh), _f32(a.q_lo), _f32(a.q_hi), _f32(a.qd_max)
            body = np.ascontiguousarray(a.sphere_body, dtype=np.int32)
            xyzr = _f32(a.sphere_xyzr)
            self._keep += [dh, lo, hi, vm, body, xyzr]
            s = self._arms[i]
            s.dof, s.n_spheres, s.K, s.H = a.dof, a.n_spheres, a.K, a.H
            s.dh, s.q_lo, s.q_hi, s.qd_max = _pf(dh), _pf(lo), _pf(hi), _pf(vm)
            s.sphere_body = body.ctypes.data_as(_ip)
            s.sphere_xyzr = _pf(xyzr)
            for k in range(7):
                s.base_pose[k] = float(a.base_pose[k])
            s.external = 1 if i in external else 0
        self.external = set(external)
        p = sc.params
        self.cfg = MrsConfig(A, self._arms, p["dt"], p["lam"], p["gamma"], p["alpha_mu"],
                             p["alpha_sigma"], p["sigma_init"], p["w_pose"], p["w_rot"],
                             p["w_stop"], p["w_joint"], p["w_coll"], p["w_self"], p["w_dyn"],
                             p["B"], p["B_world"], p["B_self"], p["tau"], p["q_margin"],
                             int(p["iterations"]), int(p["seed"]), 0,
                             int(p.get("max_plan_age", 0)), p.get("w_manip", 0.0),
                             p.get("manip_w0", 0.02))
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        h = C.c_void_p()
        st = self.L.mrs_create(C.byref(self.cfg), C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != 0:
            raise MrsError(st, "mrs_create: " + self.L.mrs_last_error(None).decode())
        self.h = h
        self.sizes = MrsSizes()
        self._check(self.L.mrs_query_sizes(self.h, C.byref(self.sizes)), "query_sizes")
        self.ws = None
        if workspace:
            nb = int(self.sizes.workspace_bytes)
            self.ws = torch.empty(nb + 256, dtype=torch.uint8, device=self.device)
            base = self.ws.data_ptr()
            off = (-base) % 256
            self._check(self.L.mrs_bind_workspace(self.h, C.c_void_p(base + off), nb), "bind")
        self.off_hd = np.concatenate([[0], np.cumsum([a.H * a.dof for a in sc.arms])]).astype(int)
        self.off_hs = np.concatenate([[0], np.cumsum([a.H * a.n_spheres * 4 for a in sc.arms])]).astype(int)
        self.off_d = np.concatenate([[0], np.cumsum([a.dof for a in sc.arms])]).astype(int)
        self.off_in = np.concatenate([[0], np.cumsum([2 * a.dof + 12 for a in sc.arms])]).astype(int)

    # -- plumbing -----------------------------------------------------------
    def _check(self, st, what):
        if st != 0:
            msg = self.L.mrs_last_error(self.h).decode() if getattr(self, "h", None) else ""
            raise MrsError(st, f"{what}: {msg}")

    def close(self):
        if getattr(self, "h", None):
            self.L.mrs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- API ----------------------------------------------------------------
    def set_world(self, spheres=None, vel=None, aabbs=None):
        """World obstacles; with no arguments, the scenario's spheres, their
        velocities (if any) and its boxes."""
        sc = self.sc
        if spheres is None:
            spheres, vel = sc.world, sc.world_vel if vel is None else vel
        spheres = _f32(spheres).reshape(-1, 4)
        vel = None if vel is None else _f32(vel).reshape(-1, 3)
        aabbs = _f32(sc.aabb if aabbs is None else aabbs).reshape(-1, 6)
        self._check(self.L.mrs_set_world(self.h, _pf(spheres) if len(spheres) else None,
                                         _pf(vel), len(spheres),
                                         _pf(aabbs) if len(aabbs) else None, len(aabbs)),
                    "set_world")

    def share_plans(self, arm, plan_spheres, plan_q, dist_to_goal, cycle):
        ps = _f32(plan_spheres)
        pq = None if plan_q is None else _f32(plan_q)
        self._check(self.L.mrs_share_plans(self.h, arm, _pf(ps), _pf(pq), float(dist_to_goal),
                                           int(cycle)), "share_plans")

    def pack_input(self, q, qd, goal_p, goal_R):
        parts = []
        for a in range(len(self.sc.arms)):
            parts += [_f32(q[a]).ravel(), _f32(qd[a]).ravel(), _f32(goal_p[a]).ravel(),
                      _f32(goal_R[a]).ravel()]
        return np.concatenate(parts).astype(np.float32)

    _OUT_KEYS = ("mean_plan", "plan_spheres", "plan_q", "u_star", "dist_to_goal", "min_cost")

    def _step_buffers(self):
        """Built once per controller: one contiguous input array (per arm q,
        qd, goal_p, goal_R) with the arm-state array pointing into it, a view
        of the context's pinned result block (mrs_output_host) and the
        slices of each output in it."""
        A = len(self.sc.arms)
        sz = self.sizes
        xin = np.zeros(sum(2 * a.dof + 12 for a in self.sc.arms), np.float32)
        states = (MrsArmState * A)()
        off = 0
        for i, a in enumerate(self.sc.arms):
            d = a.dof
            parts = (xin[off:off + d], xin[off + d:off + 2 * d], xin[off + 2 * d:off + 2 * d + 3],
                     xin[off + 2 * d + 3:off + 2 * d + 12])
            states[i] = MrsArmState(*[_pf(x) for x in parts])
            off += 2 * d + 12
        o = MrsStepOut()
        self._check(self.L.mrs_output_host(self.h, C.byref(o)), "output_host")
        ptrs = [C.cast(getattr(o, k), C.c_void_p).value for k in self._OUT_KEYS]
        base = min(ptrs)
        block = np.ctypeslib.as_array((C.c_float * int(sz.output_floats)).from_address(base))
        lens = (sz.hd, sz.hs, sz.hd, sz.d, A, A)
        keys = tuple((k, slice((p - base) // 4, (p - base) // 4 + int(n)))
                     for k, p, n in zip(self._OUT_KEYS, ptrs, lens))
        self._dofs = tuple(a.dof for a in self.sc.arms)
        self._sbuf = (xin, states, block, keys)
        return self._sbuf

    def step(self, q, qd, goal_p, goal_R):
        """One control cycle with host inputs; returns a dict of host arrays
        (fresh copies)."""
        xin, states, block, keys = getattr(self, "_sbuf", None) or self._step_buffers()
        parts = []
        for a, d in enumerate(self._dofs):
            qa, qda, gpa, gRa = q[a], qd[a], np.ravel(goal_p[a]), np.ravel(goal_R[a])
            if len(qa) != d or len(qda) != d or gpa.size != 3 or gRa.size != 9:
                raise ValueError(f"arm {a}: q, qd need {d} values, goal_p 3, goal_R 9")
            parts += (qa, qda, gpa, gRa)
        np.concatenate(parts, out=xin)
        st = self.L.mrs_step(self.h, states, None)   # results stay in the pinned block
        if st != 0:
            self._check(st, "step")
        oc = block.copy()
        return {k: oc[s] for k, s in keys}

    def step_device(self, d_input):
        """Enqueue one cycle with a device-resident packed input (torch float32
        tensor of input_floats elements); does not wait."""
        self._check(self.L.mrs_step_device(self.h, C.c_void_p(d_input.data_ptr())), "step_device")

    def output_pointers(self):
        o = MrsStepOut()
        self._check(self.L.mrs_output_device(self.h, C.byref(o)), "output_device")
        return o

    def sync(self, timeout_s=10.0):
        self._check(self.L.mrs_sync(self.h, float(timeout_s)), "sync")

    def use_graph(self, on: bool):
        self._check(self.L.mrs_use_graph(self.h, 1 if on else 0), "use_graph")

    def set_zero_noise(self, on: bool):
        self._check(self.L.mrs_set_zero_noise(self.h, 1 if on else 0), "zero_noise")

    def set_wait_limit(self, polls: int):
        """Polls of the rollout's bounded wait for its plan copies (< 0: the
        default)."""
        self._check(self.L.mrs_set_wait_limit(self.h, int(polls)), "set_wait_limit")

    def enable_timing(self, on: bool):
        self._check(self.L.mrs_enable_timing(self.h, 1 if on else 0), "enable_timing")

    def kernel_times(self):
        """Durations (ms) of the last cycle's kernels in launch order."""
        n = C.c_int(64)
        ms = np.zeros(64, np.float32)
        self._check(self.L.mrs_kernel_times(self.h, _pf(ms), C.byref(n)), "kernel_times")
        return ms[:n.value].copy()

    def set_rollout_shape(self, tile_samples=32, blocks_per_sm=0, order=0):
        sh = MrsRolloutShape(tile_samples, blocks_per_sm, order, 0.0)
        self._check(self.L.mrs_set_rollout_shape(self.h, C.byref(sh)), "set_rollout_shape")

    def rollout_shape(self):
        """(tile_samples, blocks_per_sm, order) and the maximum blocks per SM."""
        sh = MrsRolloutShape()
        mx = C.c_int()
        self._check(self.L.mrs_get_rollout_shape(self.h, C.byref(sh), C.byref(mx)), "get_rollout_shape")
        return (sh.tile_samples, sh.blocks_per_sm, sh.order), mx.value

    def autotune(self, reps=5):
        """Time every rollout shape, keep the fastest; returns (best, table)
        as dicts with tile_samples, blocks_per_sm, order, cycle_ms."""
        cap = 6 * 4 * 3   # tile sizes x resident blocks (at most 4) x orders
        tab = (MrsRolloutShape * cap)()
        n = C.c_int()
        best = MrsRolloutShape()
        self._check(self.L.mrs_autotune(self.h, int(reps), tab, cap, C.byref(n), C.byref(best)),
                    "autotune")
        conv = lambda x: dict(tile_samples=x.tile_samples, blocks_per_sm=x.blocks_per_sm,
                              order=x.order, cycle_ms=float(x.cycle_ms))
        return conv(best), [conv(tab[i]) for i in range(min(n.value, cap))]

    def save_state(self) -> bytes:
        buf = (C.c_char * int(self.sizes.state_bytes))()
        self._check(self.L.mrs_save_state(self.h, buf, len(buf)), "save_state")
        return bytes(buf)

    def load_state(self, blob: bytes):
        buf = (C.c_char * len(blob)).from_buffer_copy(blob)
        self._check(self.L.mrs_load_state(self.h, buf, len(blob)), "load_state")

    def fk(self, arm, q):
        a = self.sc.arms[arm]
        q = _f32(q).reshape(-1, a.dof)
        ee = np.zeros((len(q), 12), np.float32)
        sph = np.zeros((len(q), a.n_spheres, 4), np.float32)
        self._check(self.L.mrs_fk(self.h, arm, len(q), _pf(q), _pf(ee), _pf(sph)), "fk")
        return ee, sph

    def fk_static(self, arm, q):
        """mrs_fk_static: forward kinematics staged in the library's static
        device scratch, for callers that cannot allocate device memory."""
        a = self.sc.arms[arm]
        q = _f32(q).reshape(-1, a.dof)
        ee = np.zeros((len(q), 12), np.float32)
        sph = np.zeros((len(q), a.n_spheres, 4), np.float32)
        self._check(self.L.mrs_fk_static(self.h, arm, len(q), _pf(q), _pf(ee), _pf(sph)),
                    "fk_static")
        return ee, sph

    def goal_pose(self, arm, q):
        ee, _ = self.fk(arm, q)
        return ee[0, 9:12].copy(), ee[0, :9].reshape(3, 3).copy()

    def set_self_surrogate(self, arm, net, margin=0.03):
        """Self-collision clearance of `arm` from the surrogate `net` (an MLP;
        None: exact), exact fallback below B_self + margin."""
        self._check(self.L.mrs_set_self_surrogate(self.h, arm, net.h if net is not None else None,
                                                  float(margin)), "set_self_surrogate")
        self._nets = getattr(self, "_nets", {})
        self._nets[arm] = net   # keep the network alive while the context uses it

    def self_dataset(self, arm, n, seed):
        """Device training data: (features [n][2 dof], labels [n], q [n][dof])."""
        import torch
        d = self.sc.arms[arm].dof
        x = torch.empty((n, 2 * d), dtype=torch.float32, device=self.device)
        t = torch.empty(n, dtype=torch.float32, device=self.device)
        q = torch.empty((n, d), dtype=torch.float32, device=self.device)
        self._check(self.L.mrs_self_dataset(self.h, arm, n, int(seed), C.c_void_p(x.data_ptr()),
                                            C.c_void_p(t.data_ptr()), C.c_void_p(q.data_ptr())),
                    "self_dataset")
        return x, t, q

    def self_distance(self, arm, q):
        import torch
        out = torch.empty(q.shape[0], dtype=torch.float32, device=q.device)
        self._check(self.L.mrs_self_distance(self.h, arm, q.shape[0], C.c_void_p(q.data_ptr()),
                                             C.c_void_p(out.data_ptr())), "self_distance")
        return out

    def debug_self(self, arm):
        a = self.sc.arms[arm]
        dh = np.zeros((a.H, a.K), np.float32)
        ex = np.zeros((a.H, a.K), np.float32)
        self._check(self.L.mrs_debug_self(self.h, arm, _pf(dh), _pf(ex)), "debug_self")
        return dh, ex

    def set_pair_surrogate(self, a, b, net, margin=0.03):
        """Arm-to-arm clearance of arm a to arm b's plan (b = -1: every other
        arm) from the network `net` (None: exact), exact below B + margin."""
        self._check(self.L.mrs_set_pair_surrogate(self.h, a, b, net.h if net is not None else None,
                                                  float(margin)), "set_pair_surrogate")
        self._nets = getattr(self, "_nets", {})
        self._nets[("pair", a, b)] = net

    def relative_pose(self, a, b):
        out = np.zeros(7, np.float32)
        self._check(self.L.mrs_relative_pose(self.h, a, b, _pf(out)), "relative_pose")
        return out

    def pair_dataset(self, a, b, n, seed, poses=None, jit_t=0.02, jit_yaw=0.05):
        """Device training data of the arm-pair network: (features [n][2 d_a +
        2 d_b + 7], exact clearance [n], q_a [n][d_a], q_b [n][d_b], pose [n][7])."""
        import torch
        da, db = self.sc.arms[a].dof, self.sc.arms[b].dof
        dev = self.device
        x = torch.empty((n, 2 * da + 2 * db + 7), dtype=torch.float32, device=dev)
        t = torch.empty(n, dtype=torch.float32, device=dev)
        qa = torch.empty((n, da), dtype=torch.float32, device=dev)
        qb = torch.empty((n, db), dtype=torch.float32, device=dev)
        po = torch.empty((n, 7), dtype=torch.float32, device=dev)
        p = None if poses is None else _f32(poses).reshape(-1, 7)
        self._check(self.L.mrs_pair_dataset(
            self.h, a, b, n, seed, _pf(p) if p is not None else None,
            0 if p is None else len(p), float(jit_t), float(jit_yaw),
            C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()), C.c_void_p(qa.data_ptr()),
            C.c_void_p(qb.data_ptr()), C.c_void_p(po.data_ptr())), "pair_dataset")
        return x, t, qa, qb, po

    def debug_pair(self, a, b, predicted=True):
        """(predicted, exact) clearance [H_a][K_a] of arm a's rollout steps to
        arm b's plan in the last cycle; predicted is None when not asked."""
        A = self.sc.arms[a]
        rh = np.zeros((A.H, A.K), np.float32) if predicted else None
        ex = np.zeros((A.H, A.K), np.float32)
        self._check(self.L.mrs_debug_pair(self.h, a, b, _pf(rh) if predicted else None, _pf(ex)),
                    "debug_pair")
        return rh, ex

    def debug_costs(self, arm):
        c = np.zeros(self.sc.arms[arm].K, np.float32)
        self._check(self.L.mrs_debug_costs(self.h, arm, _pf(c)), "debug_costs")
        return c

    def debug_alpha(self):
        A = len(self.sc.arms)
        al = np.zeros((A, A), np.float32)
        self._check(self.L.mrs_debug_alpha(self.h, _pf(al)), "debug_alpha")
        return al

    def debug_spheres(self, anh):
        anh = np.ascontiguousarray(np.asarray(anh, dtype=np.int32).reshape(-1, 3))
        out = np.zeros((len(anh), MAX_SPHERES, 4), np.float32)
        self._check(self.L.mrs_debug_spheres(self.h, len(anh), anh.ctypes.data_as(_ip), _pf(out)),
                    "debug_spheres")
        return out

    def split(self, flat, kind, arm):
        a = self.sc.arms[arm]
        if kind == "hd":
            return flat[self.off_hd[arm]:self.off_hd[arm + 1]].reshape(a.H, a.dof)
        if kind == "hs":
            return flat[self.off_hs[arm]:self.off_hs[arm + 1]].reshape(a.H, a.n_spheres, 4)
        if kind == "d":
            return flat[self.off_d[arm]:self.off_d[arm + 1]]
        raise KeyError(kind)


def state_blob(sc, mu, Sigma, cycle, world_t, plan_valid, plan_stamp, plan_dist, plan_spheres,
               plan_q) -> bytes:
    """Serialise a controller state (per-arm concatenated arrays) in the layout
    of mrs_save_state / mrs_load_state."""
    import struct
    A = len(sc.arms)
    parts = [struct.pack("<IIIIqff", 0x3152534D, 1, A, 0, int(cycle), float(world_t), 0.0)]
    o_hd = o_hdd = 0
    for a in sc.arms:
        hd, hdd = a.H * a.dof, a.H * a.dof * a.dof
        parts.append(np.asarray(mu[o_hd:o_hd + hd], np.float32).tobytes())
        parts.append(np.asarray(Sigma[o_hdd:o_hdd + hdd], np.float32).tobytes())
        o_hd += hd
        o_hdd += hdd
    o_hd = o_hs = 0
    for i, a in enumerate(sc.arms):
        hd, hs = a.H * a.dof, a.H * a.n_spheres * 4
        parts.append(struct.pack("<iiqff", int(plan_valid[i]), 0, int(plan_stamp[i]),
                                 float(plan_dist[i]), 0.0))
        parts.append(np.asarray(plan_spheres[o_hs:o_hs + hs], np.float32).tobytes())
        parts.append(np.asarray(plan_q[o_hd:o_hd + hd], np.float32).tobytes())
        o_hd += hd
        o_hs += hs
    return b"".join(parts)


def selftest_gemm(A_bits, B_bits):
    """C = A B^T on the tensor cores, for BF16 bit patterns A [M][K], B [N][K]."""
    L = load()
    A_bits = np.ascontiguousarray(A_bits, dtype=np.uint16)
    B_bits = np.ascontiguousarray(B_bits, dtype=np.uint16)
    M, K = A_bits.shape
    N = B_bits.shape[0]
    C_ = np.zeros((M, N), np.float32)
    p16 = C.POINTER(C.c_uint16)
    st = L.mrs_selftest_gemm(M, N, K, A_bits.ctypes.data_as(p16), B_bits.ctypes.data_as(p16),
                             _pf(C_))
    if st != 0:
        raise MrsError(st, "selftest_gemm")
    return C_


class MLP:
    """A clearance-surrogate network on the device (mrs_mlp_*).  Inputs and
    targets are torch float32 CUDA tensors."""

    def __init__(self, in_dim, width=256, layers=3, seed=0, stream=None):
        import torch
        self.L = load()
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = C.c_void_p()
        st = self.L.mrs_mlp_create(in_dim, width, layers, seed, C.c_void_p(self.stream.cuda_stream),
                                   C.byref(h))
        if st != 0:
            raise MrsError(st, "mrs_mlp_create")
        self.h = h
        self.in_dim, self.width, self.layers = in_dim, width, layers
        n = C.c_size_t()
        self.L.mrs_mlp_param_count(self.h, C.byref(n))
        self.n_params = n.value

    def _check(self, st, what):
        if st != 0:
            raise MrsError(st, f"{what}: {self.L.mrs_mlp_last_error(self.h).decode()}")

    def set_loss(self, over_weight=1.0):
        """Weight of over-predictions in the training loss (1: plain MSE)."""
        self._check(self.L.mrs_mlp_set_loss(self.h, float(over_weight)), "set_loss")

    def launch_info(self):
        """Fused inference launch shape: CTAs per SM (plain rows, rollout
        trajectories), ring slots, shared memory per CTA, SMs."""
        info = (C.c_int * 5)()
        self._check(self.L.mrs_mlp_launch_info(self.h, info, 5), "launch_info")
        return dict(per_sm_rows=info[0], per_sm_traj=info[1], slots=info[2], smem=info[3],
                    sms=info[4])

    def close(self):
        if getattr(self, "h", None):
            self.L.mrs_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        p = np.zeros(self.n_params, np.float32)
        self._check(self.L.mrs_mlp_get_params(self.h, _pf(p), self.n_params), "get_params")
        return p

    def set_params(self, p):
        p = _f32(p)
        self._check(self.L.mrs_mlp_set_params(self.h, _pf(p), len(p)), "set_params")

    def forward(self, x):
        import torch
        y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        self._check(self.L.mrs_mlp_forward(self.h, C.c_void_p(x.data_ptr()), x.shape[0],
                                           C.c_void_p(y.data_ptr())), "forward")
        return y

    def grads(self, x, t):
        g = np.zeros(self.n_params, np.float32)
        loss = np.zeros(1, np.float32)
        self._check(self.L.mrs_mlp_grads(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()),
                                         x.shape[0], _pf(g), _pf(loss)), "grads")
        return g, float(loss[0])

    def train_step(self, x, t, lr):
        loss = np.zeros(1, np.float32)
        self._check(self.L.mrs_mlp_train_step(self.h, C.c_void_p(x.data_ptr()),
                                              C.c_void_p(t.data_ptr()), x.shape[0], float(lr),
                                              _pf(loss)), "train_step")
        return float(loss[0])

    def unpack(self, p):
        """Split a flat parameter vector into [(W, b), ...], (w_out, b_out)."""
        out, o = [], 0
        in_pad = (self.in_dim + 15) // 16 * 16
        for l in range(self.layers):
            fan = in_pad if l == 0 else self.width
            W = p[o:o + self.width * fan].reshape(self.width, fan)
            o += self.width * fan
            b = p[o:o + self.width]
            o += self.width
            out.append((W, b))
        return out, (p[o:o + self.width], p[o + self.width:o + self.width + 1])
