"""ctypes binding of liblsn (include/lsn.h).

Argument marshalling only: every function here converts Python / numpy /
torch arguments into the plain pointers and sizes of the C ABI and calls the
function of the same name.  Device tensors are passed by their data pointer;
numpy arrays by their host pointer.  The library must be built first
(``paper_2409_03807_gb300.build.build()``); loading fails loudly otherwise.
"""
import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "liblsn.so")

LSN_OK, LSN_NOT_CONVERGED, LSN_LS_FAILED, LSN_NOT_SPD, LSN_PRECISION_FLOOR = 0, 1, 2, 3, 4
LSN_SADDLE = 5
OPTIMIZERS = {"newton": 0, "lbfgs": 1}
LSN_ERR_ARG, LSN_ERR_CUDA, LSN_ERR_NONFINITE, LSN_ERR_STATE, LSN_ERR_OOM = -1, -2, -3, -4, -5
PRECISIONS = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}


class LsnStats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("ls_trials", ctypes.c_int),
                ("exit", ctypes.c_int), ("grad_inf", ctypes.c_double),
                ("energy", ctypes.c_double), ("ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LsnError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"liblsn error {code}: {msg}")
        self.code = code


_lib = None

_SIGS = {
    "lsn_create": [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p],
    "lsn_destroy": [ctypes.c_void_p],
    "lsn_last_error": [ctypes.c_void_p],
    "lsn_set_mesh": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int],
    "lsn_set_material": [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                         ctypes.c_void_p],
    "lsn_set_constraints": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "lsn_set_cubature": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int],
    "lsn_set_ground": [ctypes.c_void_p, ctypes.c_double, ctypes.c_double],
    "lsn_set_decoder": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                        ctypes.c_void_p, ctypes.c_double, ctypes.c_int],
    "lsn_set_solver": [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                       ctypes.c_double],
    "lsn_set_optimizer": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int],
    "lsn_set_exact_hessian": [ctypes.c_void_p, ctypes.c_int, ctypes.c_double],
    "lsn_selftest_bounded_wait": [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p],
    "lsn_set_affine_modes": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "lsn_tet_forces": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "lsn_select_cubature": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                            ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                            ctypes.c_void_p],
    "lsn_fullspace_setup": [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int],
    "lsn_fullspace_set_state": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "lsn_fullspace_step": [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                           ctypes.POINTER(LsnStats), ctypes.POINTER(ctypes.c_longlong)],
    "lsn_set_state": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "lsn_set_dynamics": [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p],
    "lsn_step": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                 ctypes.POINTER(LsnStats)],
    "lsn_get_positions": [ctypes.c_void_p, ctypes.c_void_p],
    "lsn_get_state": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "lsn_eval": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                 ctypes.c_void_p],
    "lsn_decode": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "lsn_set_profiling": [ctypes.c_void_p, ctypes.c_uint],
    "lsn_set_execution": [ctypes.c_void_p, ctypes.c_int],
    "lsn_get_trace": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                      ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)],
    "lsn_get_profile": [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                        ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)],
    "lsn_reset_profile": [ctypes.c_void_p],
    "lsn_train_init": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                       ctypes.c_void_p, ctypes.c_int],
    "lsn_train_num_params": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)],
    "lsn_train_get_params": [ctypes.c_void_p, ctypes.c_void_p],
    "lsn_train_set_params": [ctypes.c_void_p, ctypes.c_void_p],
    "lsn_train_get_adam": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.POINTER(ctypes.c_longlong)],
    "lsn_train_set_adam": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.c_longlong],
    "lsn_train_eval": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                       ctypes.c_void_p, ctypes.c_void_p],
    "lsn_train_step": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                       ctypes.c_double, ctypes.c_void_p],
    "lsn_train_hessians": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "lsn_set_lipschitz_order": [ctypes.c_void_p, ctypes.c_int],
    "lsn_train_eval_unsup": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                             ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                             ctypes.c_void_p],
    "lsn_train_step_unsup": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                             ctypes.c_void_p],
    "lsn_train_apply": [ctypes.c_void_p],
    "lsn_element_system_noalloc": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_void_p, ctypes.c_void_p],
}

KERNEL_CLASSES = ["decoder_hidden", "decoder_last", "element", "decoder_trial",
                  "element_energy", "solve"]


def load(path=None):
    """Load liblsn.so and declare the C signatures (raises if missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"liblsn.so not built ({path}); run "
                          "paper_2409_03807_gb300.build.build() on a machine with nvcc")
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.lsn_destroy.restype = None
    lib.lsn_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def _ptr(a):
    """Pointer of a numpy array, a torch tensor (host or device) or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _f64(a):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=np.int32)


def element_system_noalloc(S, r, n, tets, dminv, wvol, u, J, mu, lam, out, stream=None):
    """Allocation-free elastic reduced system (see include/lsn.h): all array
    arguments are device tensors; returns the C status."""
    lib = load()
    st = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    return lib.lsn_element_system_noalloc(int(S), int(r), int(n), _ptr(tets), _ptr(dminv),
                                          _ptr(wvol), _ptr(u), _ptr(J), float(mu), float(lam),
                                          _ptr(out), st)


class Context:
    """One liblsn context; methods are the C ABI calls without the prefix."""

    def __init__(self, device=0, stream=None):
        self.lib = load()
        h = ctypes.c_void_p()
        st = None if stream is None else int(getattr(stream, "cuda_stream", stream))
        rc = self.lib.lsn_create(ctypes.byref(h), int(device), st)
        if rc != 0:
            raise LsnError(rc, "lsn_create failed")
        self.h = h
        self.r = None
        self.r_nn = None
        self.affine = False
        self.n = None
        self.ne = None

    def close(self):
        if self.h:
            self.lib.lsn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self):
        return self.lib.lsn_last_error(self.h).decode()

    def _check(self, rc, allow_positive=False):
        if rc < 0 or (rc > 0 and not allow_positive):
            raise LsnError(rc, self.last_error())
        return rc

    def set_mesh(self, X0, tets):
        X0 = _f64(X0)
        tets = _i32(tets)
        self.keep = (X0, tets)
        self.n = 3 * X0.shape[0]
        self.ne = int(tets.shape[0])
        return self._check(self.lib.lsn_set_mesh(self.h, _ptr(X0), X0.shape[0], _ptr(tets),
                                                 tets.shape[0]))

    def set_material(self, youngs, poisson, density, gravity):
        g = _f64(gravity)
        return self._check(self.lib.lsn_set_material(self.h, youngs, poisson, density, _ptr(g)))

    def set_constraints(self, vidx, targets):
        vidx = _i32(vidx)
        targets = _f64(targets)
        nc = 0 if vidx is None else int(vidx.shape[0])
        if vidx is None:
            nc = int(targets.shape[0]) if targets is not None else 0
        return self._check(self.lib.lsn_set_constraints(self.h, _ptr(vidx), nc, _ptr(targets)))

    def set_cubature(self, idx, w):
        idx = _i32(idx)
        w = _f64(w)
        s = 0 if idx is None else int(idx.shape[0])
        return self._check(self.lib.lsn_set_cubature(self.h, _ptr(idx), _ptr(w), s))

    def set_ground(self, height, stiffness):
        return self._check(self.lib.lsn_set_ground(self.h, height, stiffness))

    def set_decoder(self, Ws, bs, out_scale, precision="fp32"):
        Ws = [np.ascontiguousarray(W, dtype=np.float32) for W in Ws]
        bs = [np.ascontiguousarray(b, dtype=np.float32) for b in bs]
        widths = [Ws[0].shape[1]] + [W.shape[0] for W in Ws]
        wa = (ctypes.c_int * len(widths))(*widths)
        Wp = (ctypes.c_void_p * len(Ws))(*[W.ctypes.data for W in Ws])
        bp = (ctypes.c_void_p * len(bs))(*[b.ctypes.data for b in bs])
        self.r_nn = widths[0]
        self.r = widths[0] + (12 if self.affine else 0)  # the library keeps the affine flag
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        return self._check(self.lib.lsn_set_decoder(self.h, len(Ws), wa, Wp, bp,
                                                    float(out_scale), prec))

    def set_solver(self, tol_inf, max_newton=1024, max_ls=128, armijo_c=1e-4):
        return self._check(self.lib.lsn_set_solver(self.h, tol_inf, max_newton, max_ls,
                                                   armijo_c))

    def set_affine_modes(self, center=None):
        """12 affine coordinates appended to z (center: 3 floats), or off (None)."""
        c = None if center is None else _f64(center)
        self._check(self.lib.lsn_set_affine_modes(self.h, 0 if center is None else 1, _ptr(c)))
        self.affine = center is not None
        self.r = self.r_nn + (12 if self.affine else 0)

    def tet_forces(self, Z, A=None):
        """Per-tet reduced elastic forces at the points Z (K x r): (K r) x ne."""
        Z = _f64(Z)
        K = int(Z.shape[0])
        if A is None:
            A = np.zeros((K * self.r, self.ne))
        self._check(self.lib.lsn_tet_forces(self.h, _ptr(Z), K, _ptr(A)))
        return A

    def select_cubature(self, Z, S):
        """Optimised cubature for the points Z (K x r): (tet indices, weights,
        relative residual of the force fit)."""
        Z = _f64(Z)
        idx = np.zeros(S, np.int32)
        w = np.zeros(S)
        cnt = ctypes.c_int()
        rel = np.zeros(1)
        self._check(self.lib.lsn_select_cubature(self.h, _ptr(Z), int(Z.shape[0]), int(S),
                                                 _ptr(idx), _ptr(w), ctypes.byref(cnt),
                                                 _ptr(rel)))
        k = cnt.value
        return idx[:k].copy(), w[:k].copy(), float(rel[0])

    def fullspace_setup(self, precision="fp64", cg_rtol=1e-4, max_cg=4096):
        """Full-space comparison solve: element math "fp64" or "fp32"."""
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        return self._check(self.lib.lsn_fullspace_setup(self.h, prec, float(cg_rtol),
                                                        int(max_cg)))

    def fullspace_set_state(self, q=None, v=None):
        q, v = _f64(q), _f64(v)
        return self._check(self.lib.lsn_fullspace_set_state(self.h, _ptr(q), _ptr(v)))

    def fullspace_step(self, dt=0.0, q_out=None):
        """Returns (exit status, stats dict with "cg_iters", q_out)."""
        if q_out is None:
            q_out = np.zeros(self.n)
        st = LsnStats()
        cg = ctypes.c_longlong()
        rc = self.lib.lsn_fullspace_step(self.h, float(dt), _ptr(q_out), ctypes.byref(st),
                                         ctypes.byref(cg))
        self._check(rc, allow_positive=True)
        d = st.as_dict()
        d["cg_iters"] = int(cg.value)
        return rc, d, q_out

    def set_optimizer(self, kind="newton", history=10):
        """kind: "newton" (projective Newton) or "lbfgs"; history: L-BFGS pairs."""
        return self._check(self.lib.lsn_set_optimizer(self.h, OPTIMIZERS[kind], history))

    def selftest_bounded_wait(self, seconds=0.05):
        """Run one bounded mbarrier wait that nothing completes; returns the
        error code the wait recorded (1 when it ran out)."""
        code = ctypes.c_int(0)
        self._check(self.lib.lsn_selftest_bounded_wait(self.h, float(seconds),
                                                       ctypes.byref(code)))
        return code.value

    def set_exact_hessian(self, enable=True, clamp=1e-10):
        """Projective Newton with the exact-form reduced Hessian (the decoder's
        curvature added back, then the r x r sum projected)."""
        return self._check(self.lib.lsn_set_exact_hessian(self.h, int(bool(enable)),
                                                          float(clamp)))

    def set_state(self, z=None, q=None, v=None):
        z, q, v = _f64(z), _f64(q), _f64(v)
        return self._check(self.lib.lsn_set_state(self.h, _ptr(z), _ptr(q), _ptr(v)))

    def set_dynamics(self, dt, qbar=None):
        qbar = _f64(qbar)
        return self._check(self.lib.lsn_set_dynamics(self.h, dt, _ptr(qbar)))

    def step(self, z_in=None, dt=0.0, z_out=None):
        """Returns (exit status, stats dict, z_out)."""
        z_in = _f64(z_in)
        if z_out is None:
            z_out = np.zeros(self.r)
        st = LsnStats()
        rc = self.lib.lsn_step(self.h, _ptr(z_in), float(dt), _ptr(z_out), ctypes.byref(st))
        self._check(rc, allow_positive=True)
        return rc, st.as_dict(), z_out

    def get_state(self, z=None, q=None, v=None):
        """Copy z, q, v into the given arrays / tensors (new numpy arrays if None)."""
        z = np.zeros(self.r) if z is None else z
        q = np.zeros(self.n) if q is None else q
        v = np.zeros(self.n) if v is None else v
        self._check(self.lib.lsn_get_state(self.h, _ptr(z), _ptr(q), _ptr(v)))
        return z, q, v

    def get_positions(self, out=None):
        if out is None:
            out = np.zeros(self.n)
        self._check(self.lib.lsn_get_positions(self.h, _ptr(out)))
        return out

    def eval(self, z, want_K=True):
        """E, g, K at z (K None when want_K is False: with the L-BFGS optimiser
        E and g then come from its gradient-only pass)."""
        z = _f64(z)
        E = np.zeros(1)
        g = np.zeros(self.r)
        K = np.zeros((self.r, self.r)) if want_K else None
        self._check(self.lib.lsn_eval(self.h, _ptr(z), _ptr(E), _ptr(g),
                                      _ptr(K) if want_K else None))
        return float(E[0]), g, K

    def get_trace(self, max_entries=128):
        """Per-iteration (grad_inf, energy, grad_scale, alpha) of the last step."""
        g, e, gs, a = (np.zeros(max_entries) for _ in range(4))
        cnt = ctypes.c_int()
        self._check(self.lib.lsn_get_trace(self.h, max_entries, _ptr(g), _ptr(e), _ptr(gs),
                                           _ptr(a), ctypes.byref(cnt)))
        k = cnt.value
        return {"grad_inf": g[:k], "energy": e[:k], "grad_scale": gs[:k], "alpha": a[:k]}

    def set_execution(self, mode):
        """'graph' (0, default) or 'host' (1)."""
        m = {"graph": 0, "host": 1}.get(mode, mode)
        return self._check(self.lib.lsn_set_execution(self.h, int(m)))

    def set_profiling(self, classes=()):
        mask = 0
        for c in classes:
            mask |= 1 << (KERNEL_CLASSES.index(c) if isinstance(c, str) else int(c))
        return self._check(self.lib.lsn_set_profiling(self.h, mask))

    def get_profile(self):
        """{class: (launches, timed_launches, ms_total)}"""
        out = {}
        for k, name in enumerate(KERNEL_CLASSES):
            a, b, ms = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_double()
            self._check(self.lib.lsn_get_profile(self.h, k, ctypes.byref(a), ctypes.byref(b),
                                                 ctypes.byref(ms)))
            out[name] = (a.value, b.value, ms.value)
        return out

    def reset_profile(self):
        return self._check(self.lib.lsn_reset_profile(self.h))

    # -- training (lsn_train_*) -----------------------------------------
    def train_init(self, enc_W, enc_b, tet_idx, w):
        enc_W = np.ascontiguousarray(enc_W, dtype=np.float32)
        enc_b = np.ascontiguousarray(enc_b, dtype=np.float32)
        tet_idx = _i32(tet_idx)
        w = _f64(w)
        self.keep_train = (enc_W, enc_b, tet_idx, w)
        return self._check(self.lib.lsn_train_init(self.h, _ptr(enc_W), _ptr(enc_b),
                                                   _ptr(tet_idx), _ptr(w), tet_idx.shape[0]))

    def train_num_params(self):
        n = ctypes.c_longlong()
        self._check(self.lib.lsn_train_num_params(self.h, ctypes.byref(n)))
        return n.value

    def train_get_params(self, out=None):
        out = np.zeros(self.train_num_params()) if out is None else out
        self._check(self.lib.lsn_train_get_params(self.h, _ptr(out)))
        return out

    def train_set_params(self, theta):
        theta = theta if hasattr(theta, "data_ptr") else np.ascontiguousarray(theta, np.float64)
        return self._check(self.lib.lsn_train_set_params(self.h, _ptr(theta)))

    def train_checkpoint(self):
        """Everything training needs to resume: parameters, Adam moments and
        step count (a dict of numpy arrays; np.savez(path, **ckpt) stores it)."""
        npar = self.train_num_params()
        m, v = np.zeros(npar), np.zeros(npar)
        step = ctypes.c_longlong()
        self._check(self.lib.lsn_train_get_adam(self.h, _ptr(m), _ptr(v), ctypes.byref(step)))
        return {"theta": self.train_get_params(), "adam_m": m, "adam_v": v,
                "adam_step": np.array(step.value, np.int64)}

    def train_restore(self, ckpt):
        """Inverse of train_checkpoint (after train_init with the same shapes).
        Raises ValueError when an array's length is not the network's
        parameter count (a checkpoint of another network shape)."""
        npar = self.train_num_params()
        for key in ("theta", "adam_m", "adam_v"):
            size = int(np.prod(np.shape(ckpt[key])))
            if size != npar:
                raise ValueError(f"checkpoint {key} has {size} values; this network has "
                                 f"{npar} parameters")
        self.train_set_params(ckpt["theta"])
        m, v = _f64(ckpt["adam_m"]), _f64(ckpt["adam_v"])
        return self._check(self.lib.lsn_train_set_adam(self.h, _ptr(m), _ptr(v),
                                                       int(ckpt["adam_step"])))

    def train_eval(self, q, lambda_ls, grad=None, want_grad=True):
        """(L_C, L_LS, L), gradient (numpy float64 unless `grad` is given)."""
        q = _f64(q)
        B = int(q.shape[0])
        losses = np.zeros(3)
        if grad is None and want_grad:
            grad = np.zeros(self.train_num_params())
        self._check(self.lib.lsn_train_eval(self.h, _ptr(q), B, float(lambda_ls),
                                            _ptr(losses), _ptr(grad)))
        return tuple(losses), grad

    def train_step(self, q, lambda_ls, lr):
        q = _f64(q)
        losses = np.zeros(3)
        self._check(self.lib.lsn_train_step(self.h, _ptr(q), int(q.shape[0]), float(lambda_ls),
                                            float(lr), _ptr(losses)))
        return tuple(losses)

    def train_eval_unsup(self, Z, lam, sigma, lambda_ls=0.0, grad=None, want_grad=True):
        """Eq. 4 (+ lambda_ls Eq. 9) at the samples Z (B x r):
        (L_P, L_R, L_U, L_LS, L), gradient of L."""
        Z = _f64(Z)
        losses = np.zeros(5)
        if grad is None and want_grad:
            grad = np.zeros(self.train_num_params())
        self._check(self.lib.lsn_train_eval_unsup(self.h, _ptr(Z), int(Z.shape[0]), float(lam),
                                                  float(sigma), float(lambda_ls), _ptr(losses),
                                                  _ptr(grad)))
        return tuple(losses), grad

    def train_step_unsup(self, Z, lam, sigma, lr, lambda_ls=0.0):
        Z = _f64(Z)
        losses = np.zeros(5)
        self._check(self.lib.lsn_train_step_unsup(self.h, _ptr(Z), int(Z.shape[0]), float(lam),
                                                  float(sigma), float(lambda_ls), float(lr),
                                                  _ptr(losses)))
        return tuple(losses)

    def set_lipschitz_order(self, order):
        return self._check(self.lib.lsn_set_lipschitz_order(self.h, int(order)))

    def train_hessians(self, Z):
        Z = np.ascontiguousarray(Z, np.float64)
        B, r = Z.shape
        H = np.zeros((B, r, r))
        self._check(self.lib.lsn_train_hessians(self.h, _ptr(Z), B, _ptr(H)))
        return H

    def train_apply(self):
        return self._check(self.lib.lsn_train_apply(self.h))

    def decode(self, z, want_J=True):
        z = _f64(z)
        x = np.zeros(self.n)
        J = np.zeros((self.n, self.r)) if want_J else None
        self._check(self.lib.lsn_decode(self.h, _ptr(z), _ptr(x), _ptr(J)))
        return x, J
