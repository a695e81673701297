"""Thin Python binding of libdnnmg (argument marshalling only).

Every computation runs in the CUDA library behind the C ABI declared in
include/dnnmg.h; this module converts torch tensors into device pointers and
status codes into exceptions.  It fails loudly when the library is missing.
"""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdnnmg.so")

OK, ERR_ARG, ERR_CUDA, ERR_NOT_CONVERGED, ERR_NUMERICAL, ERR_TIMEOUT, ERR_STATE = range(7)
STAGES = ("vanka_pass", "vanka_setup", "apply", "defect", "transfer", "coarse_factor",
          "coarse_solve", "krylov", "residual64", "network", "train", "vcycle")
FP64, MIXED = 0, 1
PLAIN, NET = 0, 1

c_double, c_int32, c_void_p = ctypes.c_double, ctypes.c_int32, ctypes.c_void_p


class Config(ctypes.Structure):
    """Mirror of dnnmg_config."""
    _fields_ = [("nu", c_double), ("dt", c_double), ("theta", c_double), ("alpha0", c_double),
                ("newton_tol", c_double), ("gmres_rtol", c_double), ("omega", c_double),
                ("eps_damp", c_double), ("obstacle_i0", c_int32), ("obstacle_j0", c_int32),
                ("level_solve", c_int32), ("level_coarse", c_int32), ("replaced_levels", c_int32),
                ("precision", c_int32), ("newton_max", c_int32), ("gmres_m", c_int32),
                ("gmres_maxit", c_int32), ("nu1", c_int32), ("nu2", c_int32), ("hidden", c_int32),
                ("gru_layers", c_int32), ("mlp_width", c_int32), ("fallback_newton_its", c_int32),
                ("train_batch", c_int32), ("train_seq", c_int32), ("coarse_refresh", c_int32),
                ("persistent_vcycle", c_int32), ("precond_lag", c_int32),
                ("persistent_mode", c_int32), ("lps_mode", c_int32), ("stream_pass", c_int32),
                ("net_bias", c_int32), ("net_inputs", c_int32), ("obstacle_level", c_int32)]


class StepStats(ctypes.Structure):
    """Mirror of dnnmg_step_stats."""
    _fields_ = [("newton_its", c_int32), ("gmres_its", c_int32), ("fallback", c_int32),
                ("status", c_int32), ("res0", c_double), ("res_final", c_double), ("ms", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class DnnmgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dnnmg error {code}: {msg}")
        self.code = code


_lib = None


def _declare(lib):
    P = c_void_p
    sig = {
        "dnnmg_default_config": ([P], ctypes.c_int),
        "dnnmg_setup": ([P, P, P], ctypes.c_int),
        "dnnmg_destroy": ([P], ctypes.c_int),
        "dnnmg_last_error": ([P], ctypes.c_char_p),
        "dnnmg_level_dims": ([P, ctypes.c_int, P, P], ctypes.c_int),
        "dnnmg_get_state": ([P, P], ctypes.c_int),
        "dnnmg_set_state": ([P, P], ctypes.c_int),
        "dnnmg_linearize": ([P, P], ctypes.c_int),
        "dnnmg_apply": ([P, ctypes.c_int, P, P, ctypes.c_int], ctypes.c_int),
        "dnnmg_vcycle": ([P, ctypes.c_int, P, P, ctypes.c_int], ctypes.c_int),
        "dnnmg_residual": ([P, P, P, P], ctypes.c_int),
        "dnnmg_step": ([P, ctypes.c_int, P], ctypes.c_int),
        "dnnmg_num_params": ([P], ctypes.c_size_t),
        "dnnmg_net_dims": ([P, P, P], ctypes.c_int),
        "dnnmg_set_weights": ([P, P], ctypes.c_int),
        "dnnmg_get_weights": ([P, P], ctypes.c_int),
        "dnnmg_patch_infer": ([P, P, P, P, ctypes.c_int], ctypes.c_int),
        "dnnmg_gemm_bf16": ([P, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "dnnmg_num_patches": ([P], ctypes.c_int),
        "dnnmg_set_feature_stats": ([P, P, P], ctypes.c_int),
        "dnnmg_get_fine_velocity": ([P, P], ctypes.c_int),
        "dnnmg_get_patch_inputs": ([P, P], ctypes.c_int),
        "dnnmg_train_grad": ([P, P, P, ctypes.c_int, ctypes.c_int, P, P], ctypes.c_int),
        "dnnmg_train_step": ([P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_float, P], ctypes.c_int),
        "dnnmg_reset_optimizer": ([P], ctypes.c_int),
        "dnnmg_make_sample": ([P, P, P, P, P, P], ctypes.c_int),
        "dnnmg_feature_stats": ([P, P, ctypes.c_int64, P, P], ctypes.c_int),
        "dnnmg_make_corpus": ([P, ctypes.c_int, P, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                               ctypes.c_int, P, P], ctypes.c_int),
        "dnnmg_step_io": ([P, ctypes.c_int, P, P, P], ctypes.c_int),
        "dnnmg_prolongate": ([P, ctypes.c_int, P, P], ctypes.c_int),
        "dnnmg_functionals": ([P, ctypes.c_int, P, P, P], ctypes.c_int),
        "dnnmg_relative_errors": ([P, ctypes.c_int, P, P, P], ctypes.c_int),
        "dnnmg_profile": ([P, ctypes.c_int], ctypes.c_int),
        "dnnmg_profile_read": ([P, ctypes.c_int, ctypes.c_int, P, P], ctypes.c_int),
        "dnnmg_kernel_launches": ([], ctypes.c_uint64),
        "dnnmg_vcycle_split": ([P], ctypes.c_int),
        "dnnmg_vcycle_plan": ([P, ctypes.c_int, P, P, P], ctypes.c_int),
        "dnnmg_gather_batch": ([P, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int64, P, P],
                               ctypes.c_int),
        "dnnmg_batch_setup": ([P, ctypes.c_int, P, P], ctypes.c_int),
        "dnnmg_batch_destroy": ([P], ctypes.c_int),
        "dnnmg_batch_last_error": ([P], ctypes.c_char_p),
        "dnnmg_batch_size": ([P, P, P], ctypes.c_int),
        "dnnmg_batch_layout": ([P, ctypes.c_int, P, P], ctypes.c_int),
        "dnnmg_batch_get_state": ([P, ctypes.c_int, P], ctypes.c_int),
        "dnnmg_batch_set_state": ([P, ctypes.c_int, P], ctypes.c_int),
        "dnnmg_batch_linearize": ([P], ctypes.c_int),
        "dnnmg_batch_vcycle": ([P, P, P], ctypes.c_int),
        "dnnmg_batch_vcycle_inst": ([P, ctypes.c_int, P, P], ctypes.c_int),
        "dnnmg_batch_step": ([P, ctypes.c_int, P], ctypes.c_int),
        "dnnmg_batch_set_weights": ([P, P], ctypes.c_int),
        "dnnmg_batch_set_feature_stats": ([P, P, P], ctypes.c_int),
        "dnnmg_batch_get_fine_velocity": ([P, ctypes.c_int, P], ctypes.c_int),
        "dnnmg_batch_graphs": ([P, ctypes.c_int], ctypes.c_int),
        "dnnmg_batch_profile": ([P, ctypes.c_int], ctypes.c_int),
        "dnnmg_batch_profile_read": ([P, ctypes.c_int, ctypes.c_int, P, P], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes, f.restype = args, res
    return lib


def kernel_launches():
    """Kernels launched by libdnnmg in this process so far."""
    return int(load().dnnmg_kernel_launches())


def load():
    """Load libdnnmg.so from the package directory (raises if it is absent)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        _lib = _declare(ctypes.CDLL(LIB_PATH))
    return _lib


def default_config(**overrides):
    cfg = Config()
    load().dnnmg_default_config(ctypes.byref(cfg))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


def _ptr(t):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return c_void_p(t.data_ptr())


class Context:
    """One DNN-MG solver context (wraps dnnmg_ctx)."""

    def __init__(self, cfg=None, stream=None, **overrides):
        self.lib = load()
        self.cfg = cfg if cfg is not None else default_config(**overrides)
        if cfg is not None:
            for k, v in overrides.items():
                setattr(self.cfg, k, v)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = c_void_p()
        rc = self.lib.dnnmg_setup(ctypes.byref(self.cfg), c_void_p(self.stream.cuda_stream),
                                  ctypes.byref(h))
        if rc != OK:
            raise DnnmgError(rc, self.lib.dnnmg_last_error(None).decode())
        self.h = h
        self.vdtype = torch.float64 if self.cfg.precision == FP64 else torch.float32

    def close(self):
        if getattr(self, "h", None):
            self.lib.dnnmg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != OK and rc not in allow:
            raise DnnmgError(rc, self.lib.dnnmg_last_error(self.h).decode())
        return rc

    def level_dims(self, level):
        nx, ny = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.dnnmg_level_dims(self.h, level, ctypes.byref(nx), ctypes.byref(ny)))
        return nx.value, ny.value

    def ndof(self, level):
        nx, ny = self.level_dims(level)
        return 3 * (nx + 1) * (ny + 1)

    def get_state(self):
        x = torch.empty(self.ndof(self.cfg.level_solve), dtype=torch.float64, device="cuda")
        self._check(self.lib.dnnmg_get_state(self.h, _ptr(x)))
        return x

    def set_state(self, x):
        self._check(self.lib.dnnmg_set_state(self.h, _ptr(x)))

    def linearize(self, x):
        self._check(self.lib.dnnmg_linearize(self.h, _ptr(x)))

    def apply(self, level, w, y=None):
        y = torch.empty_like(w) if y is None else y
        self._check(self.lib.dnnmg_apply(self.h, level, _ptr(w), _ptr(y), self.cfg.precision))
        return y

    def vcycle(self, level, b, x=None):
        x = torch.empty_like(b) if x is None else x
        self._check(self.lib.dnnmg_vcycle(self.h, level, _ptr(b), _ptr(x), self.cfg.precision))
        return x

    def residual(self, x, f, r=None):
        r = torch.empty_like(x) if r is None else r
        self._check(self.lib.dnnmg_residual(self.h, _ptr(x), _ptr(f), _ptr(r)))
        return r

    # -- patch network ---------------------------------------------------
    def num_params(self):
        return int(self.lib.dnnmg_num_params(self.h))

    def net_dims(self):
        ci, co = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.dnnmg_net_dims(self.h, ctypes.byref(ci), ctypes.byref(co)))
        return ci.value, co.value

    def set_weights(self, w):
        """w: host float32 array-like of num_params() values."""
        t = torch.as_tensor(w, dtype=torch.float32).contiguous().cpu()
        if t.numel() != self.num_params():
            raise ValueError("wrong parameter count")
        self._check(self.lib.dnnmg_set_weights(self.h, c_void_p(t.data_ptr())))

    def get_weights(self):
        t = torch.empty(self.num_params(), dtype=torch.float32)
        self._check(self.lib.dnnmg_get_weights(self.h, c_void_p(t.data_ptr())))
        return t

    def patch_infer(self, x_bf16, h, out=None):
        """x_bf16: cuda bfloat16 [P, C_in]; h: cuda float32 [gru_layers, P, hidden]
        (updated)."""
        P = x_bf16.shape[0]
        if h.numel() != self.cfg.gru_layers * P * self.cfg.hidden:
            raise ValueError("h must hold gru_layers x P x hidden floats")
        out = torch.empty(P, self.net_dims()[1], dtype=torch.float32, device="cuda") \
            if out is None else out
        self._check(self.lib.dnnmg_patch_infer(self.h, _ptr(x_bf16), _ptr(h), _ptr(out), P))
        return out

    def num_patches(self):
        return int(self.lib.dnnmg_num_patches(self.h))

    def set_feature_stats(self, mean, std):
        m = torch.as_tensor(mean, dtype=torch.float32).contiguous().cpu()
        s = torch.as_tensor(std, dtype=torch.float32).contiguous().cpu()
        self._check(self.lib.dnnmg_set_feature_stats(self.h, c_void_p(m.data_ptr()),
                                                     c_void_p(s.data_ptr())))

    def get_fine_velocity(self):
        nx, ny = self.level_dims(self.cfg.level_solve + self.cfg.replaced_levels)
        v = torch.empty(2 * (nx + 1) * (ny + 1), dtype=torch.float64, device="cuda")
        self._check(self.lib.dnnmg_get_fine_velocity(self.h, _ptr(v)))
        return v

    def get_patch_inputs(self):
        x = torch.empty(self.num_patches(), self.net_dims()[0], dtype=torch.bfloat16, device="cuda")
        self._check(self.lib.dnnmg_get_patch_inputs(self.h, _ptr(x)))
        return x

    def train_step(self, X, Y, B, T, lr):
        """One Adam step on a batch (X cuda bfloat16 [B,T,C_in], Y cuda float [B,T,C_out]);
        returns the loss before the update."""
        loss = ctypes.c_float()
        self._check(self.lib.dnnmg_train_step(self.h, _ptr(X), _ptr(Y), B, T, lr,
                                              ctypes.byref(loss)))
        return loss.value

    def make_sample(self, xf_prev, xf_next, X=None, Y=None):
        """Raw inputs [P, C_in] and targets [P, C_out] (cuda float) from two fine states."""
        ci, co = self.net_dims()
        P = self.num_patches()
        X = torch.empty(P, ci, dtype=torch.float32, device="cuda") if X is None else X
        Y = torch.empty(P, co, dtype=torch.float32, device="cuda") if Y is None else Y
        st = StepStats()
        self._check(self.lib.dnnmg_make_sample(self.h, _ptr(xf_prev), _ptr(xf_next), _ptr(X),
                                               _ptr(Y), ctypes.byref(st)), allow=(ERR_NOT_CONVERGED,))
        return X, Y

    def make_corpus(self, nus, spinup_steps, spinup_dt, relax_steps, T, X=None, Y=None):
        """Raw inputs [n_traj, T, P, C_in] and targets [n_traj, T, P, C_out]
        (cuda float) of plain trajectories with viscosities nus."""
        ci, co = self.net_dims()
        P, n = self.num_patches(), len(nus)
        X = torch.empty(n, T, P, ci, dtype=torch.float32, device="cuda") if X is None else X
        Y = torch.empty(n, T, P, co, dtype=torch.float32, device="cuda") if Y is None else Y
        if X.numel() != n * T * P * ci or Y.numel() != n * T * P * co:
            raise ValueError("X, Y must hold n_traj x T x P x C_in / C_out floats")
        nu = (ctypes.c_double * n)(*[float(v) for v in nus])
        self._check(self.lib.dnnmg_make_corpus(self.h, n, nu, spinup_steps, spinup_dt,
                                               relax_steps, T, _ptr(X), _ptr(Y)))
        return X, Y

    def feature_stats(self, X, rows=None):
        ci = self.net_dims()[0]
        rows = X.numel() // ci if rows is None else rows
        m = torch.empty(ci, dtype=torch.float32)
        s = torch.empty(ci, dtype=torch.float32)
        self._check(self.lib.dnnmg_feature_stats(self.h, _ptr(X), rows, c_void_p(m.data_ptr()),
                                                 c_void_p(s.data_ptr())))
        return m, s

    def gather_batch(self, X, Y, idx, T, stride):
        """idx: cuda int32 [B, 2]; returns (Xb bfloat16 [B,T,C_in], Yb float [B,T,C_out])."""
        ci, co = self.net_dims()
        B = idx.shape[0]
        Xb = torch.empty(B, T, ci, dtype=torch.bfloat16, device="cuda")
        Yb = torch.empty(B, T, co, dtype=torch.float32, device="cuda")
        self._check(self.lib.dnnmg_gather_batch(self.h, _ptr(X), _ptr(Y), _ptr(idx), B, T, stride,
                                                _ptr(Xb), _ptr(Yb)))
        return Xb, Yb

    def gemm_bf16(self, A, B):
        """C = A @ B.T on the tensor cores (A [M,K], B [N,K] cuda bfloat16)."""
        M, K = A.shape
        N = B.shape[0]
        C = torch.empty(M, N, dtype=torch.float32, device="cuda")
        self._check(self.lib.dnnmg_gemm_bf16(self.h, _ptr(A), _ptr(B), _ptr(C), M, N, K))
        return C

    def step_io(self, mode, x_in_host, x_out_host):
        """Time step with the state exchanged through host memory (CPU tensors)."""
        st = StepStats()
        pin = c_void_p(x_in_host.data_ptr()) if x_in_host is not None else None
        pout = c_void_p(x_out_host.data_ptr()) if x_out_host is not None else None
        self._check(self.lib.dnnmg_step_io(self.h, mode, pin, pout, ctypes.byref(st)),
                    allow=(ERR_NOT_CONVERGED,))
        return st.as_dict()

    def prolongate(self, level, xc):
        xf = torch.empty(self.ndof(level + 1), dtype=torch.float64, device="cuda")
        self._check(self.lib.dnnmg_prolongate(self.h, level, _ptr(xc), _ptr(xf)))
        return xf

    def _check_state(self, level, *xs):
        n = self.ndof(level)
        for t in xs:
            if t is not None and (t.dtype != torch.float64 or t.numel() != n):
                raise ValueError(f"expected {n} float64 values for level {level}")

    def functionals(self, level, x, x_old=None):
        """(J_div, J_drag, J_lift) of state x on `level` (x_old: the state one
        step earlier, None for the steady form)."""
        self._check_state(level, x, x_old)
        out = (ctypes.c_double * 3)()
        xo = _ptr(x_old) if x_old is not None else None
        self._check(self.lib.dnnmg_functionals(self.h, level, _ptr(x), xo, out))
        return tuple(out)

    def relative_errors(self, level, x, x_ref):
        """(velocity, pressure) relative l2 errors of x against x_ref."""
        self._check_state(level, x, x_ref)
        out = (ctypes.c_double * 2)()
        self._check(self.lib.dnnmg_relative_errors(self.h, level, _ptr(x), _ptr(x_ref), out))
        return tuple(out)

    def vcycle_split(self):
        return int(self.lib.dnnmg_vcycle_split(self.h))

    def vcycle_plan(self):
        """{'split_level', 'split_mode', 'pass_shapes': {level: shape}} chosen by the autotuner."""
        sl, sm, sh = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        shapes = {}
        for lev in range(1, self.cfg.level_solve + 1):
            self._check(self.lib.dnnmg_vcycle_plan(self.h, lev, ctypes.byref(sl), ctypes.byref(sm),
                                                   ctypes.byref(sh)))
            shapes[lev] = sh.value
        return {"split_level": sl.value, "split_mode": sm.value, "pass_shapes": shapes}

    def profile(self, enable=True):
        self._check(self.lib.dnnmg_profile(self.h, 1 if enable else 0))

    def profile_read(self, stage, level=-1):
        n, t = ctypes.c_int64(), ctypes.c_double()
        self._check(self.lib.dnnmg_profile_read(self.h, stage, level, ctypes.byref(n),
                                                ctypes.byref(t)))
        return n.value, t.value

    def step(self, mode=PLAIN):
        st = StepStats()
        self._check(self.lib.dnnmg_step(self.h, mode, ctypes.byref(st)), allow=(ERR_NOT_CONVERGED,))
        return st.as_dict()


def level_nodes(level):
    """Nodes (nx+1)(ny+1) of mesh level `level` of the channel."""
    return (16 * 2 ** level + 1) * (4 * 2 ** level + 1)


class Batch:
    """Many independent problems stepped in lock-step (wraps dnnmg_batch).

    cfgs: list of Config (see dnnmg_batch_setup for the fields that may differ).
    """

    def __init__(self, cfgs, stream=None):
        self.lib = load()
        self.cfgs = list(cfgs)
        arr = (Config * len(self.cfgs))(*self.cfgs)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = c_void_p()
        rc = self.lib.dnnmg_batch_setup(arr, len(self.cfgs), c_void_p(self.stream.cuda_stream),
                                        ctypes.byref(h))
        if rc != OK:
            raise DnnmgError(rc, self.lib.dnnmg_batch_last_error(None).decode())
        self.h = h
        n, length = ctypes.c_int(), ctypes.c_int64()
        self._check(self.lib.dnnmg_batch_size(self.h, ctypes.byref(n), ctypes.byref(length)))
        self.n, self.length = n.value, length.value
        self.vdtype = torch.float64 if self.cfgs[0].precision == FP64 else torch.float32

    def close(self):
        if getattr(self, "h", None):
            self.lib.dnnmg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != OK and rc not in allow:
            raise DnnmgError(rc, self.lib.dnnmg_batch_last_error(self.h).decode())
        return rc

    def layout(self, inst):
        """(finest solved level, offset in the concatenated vectors) of problem inst."""
        lev, off = ctypes.c_int(), ctypes.c_int64()
        self._check(self.lib.dnnmg_batch_layout(self.h, inst, ctypes.byref(lev), ctypes.byref(off)))
        return lev.value, off.value

    def get_state(self, inst):
        lev, _ = self.layout(inst)
        x = torch.empty(3 * level_nodes(lev), dtype=torch.float64, device="cuda")
        self._check(self.lib.dnnmg_batch_get_state(self.h, inst, _ptr(x)))
        return x

    def set_state(self, inst, x):
        self._check(self.lib.dnnmg_batch_set_state(self.h, inst, _ptr(x)))

    def linearize(self):
        self._check(self.lib.dnnmg_batch_linearize(self.h))

    def vcycle(self, b, x=None):
        """b, x: concatenated cuda vectors of `length` elements (batch precision)."""
        x = torch.empty_like(b) if x is None else x
        self._check(self.lib.dnnmg_batch_vcycle(self.h, _ptr(b), _ptr(x)))
        return x

    def vcycle_inst(self, inst, b, x=None):
        """One V-cycle of problem inst alone (b, x: its own cuda vectors)."""
        x = torch.empty_like(b) if x is None else x
        self._check(self.lib.dnnmg_batch_vcycle_inst(self.h, inst, _ptr(b), _ptr(x)))
        return x

    def step(self, mode=PLAIN):
        """One time step of every problem; returns the list of per-problem stats."""
        st = (StepStats * self.n)()
        self._check(self.lib.dnnmg_batch_step(self.h, mode, st), allow=(ERR_NOT_CONVERGED,))
        return [s.as_dict() for s in st]

    def set_weights(self, w):
        t = torch.as_tensor(w, dtype=torch.float32).contiguous().cpu()
        self._check(self.lib.dnnmg_batch_set_weights(self.h, c_void_p(t.data_ptr())))

    def set_feature_stats(self, mean, std):
        m = torch.as_tensor(mean, dtype=torch.float32).contiguous().cpu()
        s = torch.as_tensor(std, dtype=torch.float32).contiguous().cpu()
        self._check(self.lib.dnnmg_batch_set_feature_stats(self.h, c_void_p(m.data_ptr()),
                                                           c_void_p(s.data_ptr())))

    def get_fine_velocity(self, inst):
        lev, _ = self.layout(inst)
        v = torch.empty(2 * level_nodes(lev + self.cfgs[0].replaced_levels), dtype=torch.float64,
                        device="cuda")
        self._check(self.lib.dnnmg_batch_get_fine_velocity(self.h, inst, _ptr(v)))
        return v

    def graphs(self, on=True):
        self._check(self.lib.dnnmg_batch_graphs(self.h, 1 if on else 0))

    def profile(self, enable=True):
        self._check(self.lib.dnnmg_batch_profile(self.h, 1 if enable else 0))

    def profile_read(self, stage, level=-1):
        n, t = ctypes.c_int64(), ctypes.c_double()
        self._check(self.lib.dnnmg_batch_profile_read(self.h, stage, level, ctypes.byref(n),
                                                      ctypes.byref(t)))
        return n.value, t.value
