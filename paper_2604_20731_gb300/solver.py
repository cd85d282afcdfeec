"""Python binding of the hybrid IGA-ADS + CRVPINN solver (one context per
scenario).  Argument marshalling only: every step runs in libadsgb's CUDA
kernels; the names follow the C ABI in include/adsgb.h.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import _lib as L

_DT = {"f64": L.ADS_F64, "f32": L.ADS_F32, "bf16": L.ADS_BF16}


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(sc, ads_dtype: str = "f64", any_degree: bool = False) -> L.ads_params:
    """ads_params of a scenario.  The context path (ads_init) is quadratic
    (p = 2); any_degree=True is for the degree-p plans (ads_degree_*), which
    take the degree as an argument of their own."""
    if getattr(sc, "p", 2) != 2 and not any_degree:
        raise ValueError("the context path implements quadratic B-splines (p = 2); "
                         "use the degree-p plans (ads_degree_*) for p = 3, 4")
    p = L.ads_params()
    p.dim, p.n = sc.dim, sc.n
    p.phi = float(sc.phi)
    p.mu_w, p.mu_g, p.rho_w, p.rho_g = sc.mu_w, sc.mu_g, sc.rho_w, sc.rho_g
    p.grav, p.grav_sign, p.kz_ratio = sc.grav, sc.grav_sign, sc.kz_ratio
    if len(sc.sources) > L.MAX_SOURCES:
        raise ValueError("too many sources")
    p.n_src = len(sc.sources)
    for i, s in enumerate(sc.sources):
        c = list(s.center) + [0.0] * (3 - len(s.center))
        p.src[i].center[:] = c[:3]
        p.src[i].sigma, p.src[i].rate, p.src[i].kind = s.sigma, s.rate, s.kind
    p.ads_dtype = _DT[ads_dtype]
    return p


class HybridSolver:
    """One scenario resident on the GPU: saturation, pressure, network, Adam."""

    def __init__(self, sc, width: Optional[int] = 64, crv_dtype: str = "f32",
                 ads_dtype: str = "f64", stream=None, act_chunks: int = 0, allocator=None):
        self.lib = L.load()
        self.sc = sc
        if ads_dtype not in ("f64", "f32"):
            raise ValueError("ads_dtype must be f64 or f32")
        self.params = make_params(sc, ads_dtype)
        self.crv = None
        if width is not None:
            self.crv = L.crvpinn_params(width, 4, _DT[crv_dtype], int(act_chunks))
        K = np.ascontiguousarray(sc.K, dtype=np.float64)
        phi = None if sc.phi_map is None else np.ascontiguousarray(sc.phi_map, dtype=np.float64)
        S0 = np.ascontiguousarray(sc.S0_or_zero(), dtype=np.float64)
        handle = C.c_void_p()
        st = None
        if stream is not None:
            st = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        if allocator is None:
            rc = self.lib.ads_init(C.byref(self.params), C.byref(self.crv) if self.crv else None,
                                   _dptr(K), _dptr(phi) if phi is not None else None, _dptr(S0),
                                   st, C.byref(handle))
        else:
            # allocator = (alloc(bytes) -> device pointer or 0, free(pointer)); the
            # callbacks live as long as this object
            fa, ff = allocator
            self._alloc = L.ads_allocator(L.ALLOC_FN(lambda nbytes, user: fa(nbytes) or None),
                                          L.FREE_FN(lambda ptr, user: ff(ptr)), None)
            rc = self.lib.ads_init_with_allocator(C.byref(self.params),
                                                  C.byref(self.crv) if self.crv else None, _dptr(K),
                                                  _dptr(phi) if phi is not None else None, _dptr(S0),
                                                  st, C.byref(self._alloc), C.byref(handle))
        if rc != L.ADS_OK:
            raise L.AdsError(rc, "ads_init")
        self.ctx = handle
        self.n = sc.n
        self.dim = sc.dim

    # ---- helpers ----
    def _check(self, rc, where):
        if rc != L.ADS_OK:
            raise L.AdsError(rc, where, self.lib.ads_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.ads_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def count(self, field: str) -> int:
        c = C.c_size_t()
        self._check(self.lib.ads_field_count(self.ctx, L.FIELD[field], C.byref(c)), "ads_field_count")
        return c.value

    def get(self, field: str) -> np.ndarray:
        n = self.count(field)
        out = np.empty(n, dtype=np.float64)
        self._check(self.lib.ads_get(self.ctx, L.FIELD[field], _dptr(out), n), f"ads_get({field})")
        d = self.dim
        if field in ("S", "P"):
            return out.reshape((self.n + 2,) * d)
        if field in ("K", "ALPHA"):
            return out.reshape((self.n + 1,) * d)
        return out

    def device_ptr(self, field: str):
        p, c, dt = C.c_void_p(), C.c_size_t(), C.c_int()
        self._check(self.lib.ads_device_ptr(self.ctx, L.FIELD[field], C.byref(p), C.byref(c),
                                            C.byref(dt)), "ads_device_ptr")
        return p.value, c.value, dt.value

    @property
    def nparams(self) -> int:
        v = C.c_int()
        self._check(self.lib.crvpinn_num_params(self.ctx, C.byref(v)), "crvpinn_num_params")
        return v.value

    # ---- entry points ----
    def set_theta(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        if th.size != self.nparams:
            raise ValueError("theta has the wrong size")
        self._check(self.lib.crvpinn_set_theta(self.ctx, _dptr(th)), "crvpinn_set_theta")

    def set_pressure(self, P):
        a = np.ascontiguousarray(P, dtype=np.float64)
        self._check(self.lib.ads_set_pressure_coeffs(self.ctx, _dptr(a)), "ads_set_pressure_coeffs")

    def set_saturation(self, S):
        a = np.ascontiguousarray(S, dtype=np.float64)
        self._check(self.lib.ads_set_saturation(self.ctx, _dptr(a)), "ads_set_saturation")

    def saturation_step(self, dt: float, n_sub: int = 1):
        self._check(self.lib.ads_saturation_step(self.ctx, float(dt), int(n_sub)), "ads_saturation_step")

    def cfl_dt(self, cfl=0.1, src_frac=0.05, dt_cap=1e30) -> float:
        out = C.c_double()
        self._check(self.lib.ads_cfl_dt(self.ctx, cfl, src_frac, dt_cap, C.byref(out)), "ads_cfl_dt")
        return out.value

    def galerkin_pressure(self):
        """Pressure coefficients from the Galerkin system (the plain method)."""
        self._check(self.lib.ads_galerkin_pressure(self.ctx), "ads_galerkin_pressure")

    def plain_step(self, n_sub: int = 10, dt: Optional[float] = None, cfl: float = 0.1,
                   src_frac: float = 0.05, dt_cap: float = 1e30):
        """One step of the IGA-ADS + direct-solver method (Sec. 7): the Galerkin
        pressure, then n_sub explicit saturation steps with it (CFL step size
        when dt is None).  Stays on the device; returns nothing."""
        self.galerkin_pressure()
        if dt is None:
            self._check(self.lib.ads_cfl_dt(self.ctx, cfl, src_frac, dt_cap, None), "ads_cfl_dt")
            dt = 0.0
        self.saturation_step(dt, n_sub)

    def update_coefficients(self):
        self._check(self.lib.crvpinn_update_coefficients(self.ctx), "crvpinn_update_coefficients")

    def loss_grad(self) -> float:
        out = C.c_double()
        self._check(self.lib.crvpinn_loss_grad(self.ctx, C.byref(out)), "crvpinn_loss_grad")
        return out.value

    def pretrain(self, iters: int, lr: float, sync: bool = True):
        out = C.c_double()
        self._check(self.lib.crvpinn_pretrain(self.ctx, int(iters), float(lr), C.byref(out) if sync else None),
                    "crvpinn_pretrain")
        return out.value if sync else None

    def pressure_update(self, iters: int, lr: float, sync: bool = True):
        out = C.c_double()
        self._check(self.lib.crvpinn_pressure_update(self.ctx, int(iters), float(lr),
                                                     C.byref(out) if sync else None),
                    "crvpinn_pressure_update")
        return out.value if sync else None

    def project_pressure(self):
        self._check(self.lib.ads_project_pressure(self.ctx), "ads_project_pressure")

    @staticmethod
    def hybrid_params(n_sub=10, dt=1.0, dt_policy=1, cfl=0.1, src_frac=0.05, adam_iters=100,
                      lr=1e-3) -> L.hybrid_params:
        return L.hybrid_params(int(n_sub), float(dt), int(dt_policy), float(cfl), float(src_frac),
                               int(adam_iters), float(lr))

    def hybrid_step(self, hp: L.hybrid_params, stats: bool = True):
        s = L.hybrid_stats()
        self._check(self.lib.hybrid_step(self.ctx, C.byref(hp), C.byref(s) if stats else None),
                    "hybrid_step")
        if stats:
            return dict(dt_used=s.dt_used, loss_last=s.loss_last, mass_err=s.mass_err,
                        mass_total=s.mass_total)
        return None

    def save(self, path: str):
        """Write the context's evolving state to a checkpoint file."""
        self._check(self.lib.ads_save(self.ctx, str(path).encode()), "ads_save")

    def load(self, path: str):
        """Read a checkpoint written by save() from a context of the same shape."""
        self._check(self.lib.ads_load(self.ctx, str(path).encode()), "ads_load")

    def vjp(self, g_u) -> np.ndarray:
        """(du/dtheta)^T g_u for the network's values u on the interior
        collocation nodes (crvpinn_vjp); returns nparams doubles."""
        g = np.ascontiguousarray(np.asarray(g_u, dtype=np.float64).ravel())
        if g.size != self.count("U"):
            raise ValueError("one value per interior collocation node")
        out = np.empty(self.nparams)
        self._check(self.lib.crvpinn_vjp(self.ctx, _dptr(g), _dptr(out)), "crvpinn_vjp")
        return out

    def network_nodal(self) -> np.ndarray:
        """The network's values on all (N+1)^dim nodes at the current
        parameters (boundary 0), [y][x] (or [z][y][x])."""
        self.vjp(np.zeros(self.count("U")))  # runs the forward (the cotangent is zero)
        N, d = self.n, self.dim
        out = np.zeros((N + 1,) * d)
        out[(slice(1, N),) * d] = self.get("U").reshape((N - 1,) * d)
        return out

    def set_concurrency(self, contexts: int):
        """Expect `contexts` contexts on the GPU at once (launch shapes for
        throughput rather than this context's latency)."""
        self._check(self.lib.ads_set_concurrency(self.ctx, int(contexts)), "ads_set_concurrency")

    def kernel_launches(self) -> int:
        v = C.c_ulonglong()
        self._check(self.lib.ads_kernel_launches(self.ctx, C.byref(v)), "ads_kernel_launches")
        return v.value

    def profile_train(self, iters: int = 20) -> dict:
        ms = np.zeros(len(L.TRAIN_KERNELS))
        self._check(self.lib.ads_profile_train(self.ctx, int(iters), _dptr(ms)), "ads_profile_train")
        return dict(zip(L.TRAIN_KERNELS, ms.tolist()))

    def profile_saturation(self, steps: int = 10) -> dict:
        ms = np.zeros(len(L.SAT_KERNELS))
        self._check(self.lib.ads_profile_saturation(self.ctx, int(steps), _dptr(ms)),
                    "ads_profile_saturation")
        return dict(zip(L.SAT_KERNELS, ms.tolist()))

    def sync(self, timeout_s: float = 600.0):
        self._check(self.lib.ads_sync(self.ctx, timeout_s), "ads_sync")


def hybrid_step_batch(solvers, hp: L.hybrid_params, stats: bool = False):
    lib = L.load()
    arr = (C.c_void_p * len(solvers))(*[s.ctx for s in solvers])
    out = (L.hybrid_stats * len(solvers))() if stats else None
    rc = lib.hybrid_step_batch(arr, len(solvers), C.byref(hp), out)
    if rc != L.ADS_OK:
        raise L.AdsError(rc, "hybrid_step_batch")
    if stats:
        return [dict(dt_used=s.dt_used, loss_last=s.loss_last, mass_err=s.mass_err,
                     mass_total=s.mass_total) for s in out]
    return None


def pressure_network_gradient(solver, plan, K, phi, S0, dt: float, n_steps: int, lam):
    """Gradient of J = lam . S_n with respect to the network's parameters, for
    S_n the state after n_steps explicit saturation steps (plan, degree p)
    from S0 with the network pressure: the network's nodal values (solver,
    2D, N = n) projected into the plan's splines (Sec. 6, step 4).  The
    chain runs backward through the steps (steps_with_gradient), the
    projection (project_vjp) and the network (crvpinn_vjp), every part a
    hand-written adjoint.  K, phi (nullable), S0, lam: CUDA float64 tensors
    as for steps_with_gradient.  Returns S_n, dJ/dS0 (tensors), dJ/dtheta
    (nparams, numpy) and dJ/d(rate, centre x, centre y) per source."""
    import torch
    if solver.dim != 2 or solver.n != plan.n:
        raise ValueError("the network's collocation grid must be the plan's 2D mesh")
    dev = S0.device
    stream = C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    nodal = torch.from_numpy(solver.network_nodal()).to(dev)
    P = torch.empty_like(S0)
    plan.project(nodal, P, stream)
    Sn, gS0, gP, gsrc = plan.steps_with_gradient(K, phi, S0, P, dt, n_steps, lam)
    gnod = torch.empty_like(nodal)
    plan.project_vjp(gP, gnod, stream)
    g_u = gnod[1:-1, 1:-1].cpu().numpy()
    return Sn, gS0, solver.vjp(g_u), gsrc


BATCH_PROFILE_KERNELS = ("stage_fwd", "mlp_fwd", "gram_rows_residual", "gram_cols", "gram_rows_loss",
                         "adjoint_loss_finalize", "mlp_bwd", "grad_adam")


def hybrid_step_batch_profile(solvers, iters: int = 20) -> dict:
    """Average ms of each grouped kernel of one batched Adam iteration
    (hybrid_step_batch_profile); the solvers must share the grouped shape."""
    lib = L.load()
    arr = (C.c_void_p * len(solvers))(*[s.ctx for s in solvers])
    ms = (C.c_double * 8)()
    rc = lib.hybrid_step_batch_profile(arr, len(solvers), int(iters), ms)
    if rc != L.ADS_OK:
        raise L.AdsError(rc, "hybrid_step_batch_profile")
    return dict(zip(BATCH_PROFILE_KERNELS, list(ms)))


class Server:
    """Continuous-batching server (ads_server_* in the C ABI): scenarios are
    submitted as they arrive, admitted by device-memory budget, stepped in
    rounds on several streams, and collected with wait()."""

    def __init__(self, hbm_budget: int = 8 << 30, max_active: int = 64, n_streams: int = 8):
        self.lib = L.load()
        cfg = L.ads_server_config(int(hbm_budget), int(max_active), int(n_streams))
        h = C.c_void_p()
        rc = self.lib.ads_server_create(C.byref(cfg), C.byref(h))
        if rc != L.ADS_OK:
            raise L.AdsError(rc, "ads_server_create")
        self.h = h
        self._shapes = {}

    def submit(self, sc, n_steps: int, hp: L.hybrid_params, width: int = 64,
               crv_dtype: str = "bf16", ads_dtype: str = "f32", pretrain_iters: int = 300,
               pretrain_lr: float = 1e-3, theta0=None) -> int:
        spec = L.ads_request_spec()
        spec.params = make_params(sc, ads_dtype)
        spec.crv = L.crvpinn_params(width, 4, _DT[crv_dtype])
        spec.hp = hp
        spec.n_steps = int(n_steps)
        spec.pretrain_iters = int(pretrain_iters)
        spec.pretrain_lr = float(pretrain_lr)
        K = np.ascontiguousarray(sc.K, dtype=np.float64)
        phi = None if sc.phi_map is None else np.ascontiguousarray(sc.phi_map, dtype=np.float64)
        S0 = np.ascontiguousarray(sc.S0_or_zero(), dtype=np.float64)
        th = None if theta0 is None else np.ascontiguousarray(theta0, dtype=np.float64)
        rid = C.c_int64()
        rc = self.lib.ads_server_submit(self.h, C.byref(spec), _dptr(K),
                                        _dptr(phi) if phi is not None else None, _dptr(S0),
                                        _dptr(th) if th is not None else None, C.byref(rid))
        if rc != L.ADS_OK:
            raise L.AdsError(rc, "ads_server_submit")
        self._shapes[rid.value] = (sc.n + 2,) * sc.dim
        return rid.value

    def wait(self, rid: int, timeout_s: float = 600.0):
        shape = self._shapes.pop(rid)
        S = np.empty(shape)
        P = np.empty(shape)
        res = L.ads_request_result()
        rc = self.lib.ads_server_wait(self.h, int(rid), float(timeout_s), _dptr(S), _dptr(P),
                                      C.byref(res))
        if rc != L.ADS_OK:
            raise L.AdsError(rc, f"ads_server_wait({rid})")
        info = dict(steps=res.steps, queue_ms=res.queue_ms, total_ms=res.total_ms,
                    p50_step_ms=res.p50_step_ms, p99_step_ms=res.p99_step_ms,
                    dt_used=res.last.dt_used, loss_last=res.last.loss_last,
                    mass_err=res.last.mass_err, mass_total=res.last.mass_total)
        return S, P, info

    def stats(self) -> dict:
        st = L.ads_server_stats_t()
        rc = self.lib.ads_server_stats(self.h, C.byref(st))
        if rc != L.ADS_OK:
            raise L.AdsError(rc, "ads_server_stats")
        return {k: getattr(st, k) for k, _ in st._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.lib.ads_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DegreePlan:
    """A degree-p (2, 3 or 4) FP64 2D saturation plan (ads_degree_*): the
    explicit step, its vector-Jacobian product, the projection of nodal
    values, the CFL step size and the mass, on device arrays the caller owns
    (torch CUDA tensors, float64, contiguous).  Marshalling only."""

    def __init__(self, sc, degree: int):
        self.lib = L.load()
        self.n, self.p = sc.n, int(degree)
        self.params = make_params(sc, "f64", any_degree=True)
        self.n_src = self.params.n_src
        plan = C.c_void_p()
        rc = self.lib.ads_degree_plan_create(C.byref(self.params), self.p, C.byref(plan))
        if rc != L.ADS_OK:
            raise L.AdsError(rc, "ads_degree_plan_create", "")
        self.plan = plan

    @staticmethod
    def _p(t):
        return None if t is None else t.data_ptr()

    def _check(self, rc, where):
        if rc != L.ADS_OK:
            raise L.AdsError(rc, where, "")

    def step(self, K, phi, S, P, dt, out, stream=None):
        self._check(self.lib.ads_degree_step(self.plan, self._p(K), self._p(phi), self._p(S), self._p(P),
                                             float(dt), self._p(out), stream), "ads_degree_step")

    def vjp(self, K, phi, S, P, dt, lam, gS, gP, stream=None):
        """dJ/dS into gS, dJ/dP into gP for J = lam . step(S, P); returns
        dJ/d(rate, centre x, centre y) per source, shape (n_src, 3)."""
        g = (C.c_double * max(1, 3 * self.n_src))()
        self._check(self.lib.ads_degree_step_vjp(self.plan, self._p(K), self._p(phi), self._p(S), self._p(P),
                                                 float(dt), self._p(lam), self._p(gS), self._p(gP),
                                                 g if self.n_src else None, stream), "ads_degree_step_vjp")
        return np.array(g[:3 * self.n_src]).reshape(self.n_src, 3)

    def project(self, nodal, out, stream=None):
        self._check(self.lib.ads_degree_project(self.plan, self._p(nodal), self._p(out), stream),
                    "ads_degree_project")

    def project_vjp(self, g, out, stream=None):
        """The adjoint of project: dJ/d(nodal) into out ((n+1)^2) for J = g . P."""
        self._check(self.lib.ads_degree_project_vjp(self.plan, self._p(g), self._p(out), stream),
                    "ads_degree_project_vjp")

    def cfl_dt(self, K, phi, P, cfl=0.1, src_frac=0.05, dt_cap=float("inf"), stream=None):
        dt = C.c_double()
        self._check(self.lib.ads_degree_cfl_dt(self.plan, self._p(K), self._p(phi), self._p(P), float(cfl),
                                               float(src_frac), float(dt_cap), C.byref(dt), stream),
                    "ads_degree_cfl_dt")
        return dt.value

    def mass(self, S, stream=None):
        m = C.c_double()
        self._check(self.lib.ads_degree_mass(self.plan, self._p(S), C.byref(m), stream), "ads_degree_mass")
        return m.value

    def steps_with_gradient(self, K, phi, S0, P, dt, n_steps, lam):
        """n_steps explicit steps from S0 with the pressure P fixed, and the
        gradient of J = lam . S_n: the states go forward on the device, then
        the vector-Jacobian products run backward, the adjoint of each step
        becoming the next one's lam.  Returns S_n, dJ/dS0, dJ/dP (tensors)
        and dJ/d(rate, centre x, centre y) per source (the well-placement
        gradient).  Everything runs on torch's current stream."""
        import torch
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        states = [S0]
        for _ in range(n_steps):
            out = torch.empty_like(S0)
            self.step(K, phi, states[-1], P, dt, out, stream)
            states.append(out)
        adj = lam.clone()
        gP_tot = torch.zeros_like(P)
        gsrc = np.zeros((self.n_src, 3))
        gS, gP = torch.empty_like(S0), torch.empty_like(P)
        for k in range(n_steps - 1, -1, -1):
            gsrc += self.vjp(K, phi, states[k], P, dt, adj, gS, gP, stream)
            gP_tot += gP
            adj, gS = gS, adj
        return states[-1], adj, gP_tot, gsrc

    def close(self):
        if self.plan:
            self.lib.ads_degree_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def map_from_image(img, n, flip_y: bool = True, mean: str = "arithmetic", scale: float = 1.0,
                   offset: float = 0.0, out=None):
    """Nodal values on the (n+1)^d vertex grid of a porosity or permeability
    picture (ads_map_from_image): each node averages the pixel field
    offset + scale * pixel over its dual cell.

    img: a contiguous CUDA tensor, float32 or uint8, (H, W) for 2D or
    (D, H, W) for 3D; row 0 is the picture's top edge when flip_y.  n: elements
    per axis, an int or (nx, ny(, nz)).  mean: "arithmetic" or "geometric".
    Returns (or fills `out`) a float64 CUDA tensor [y][x] (or [z][y][x]).
    Runs on torch's current stream and waits for it (bounded)."""
    import torch
    lib = L.load()
    dim = img.dim()
    if dim not in (2, 3):
        raise ValueError("img must be (H, W) or (D, H, W)")
    if img.dtype == torch.float32:
        ptype = L.ADS_PIXEL_F32
    elif img.dtype == torch.uint8:
        ptype = L.ADS_PIXEL_U8
    else:
        raise TypeError("pixels must be float32 or uint8")
    if not (img.is_cuda and img.is_contiguous()):
        raise ValueError("img must be a contiguous CUDA tensor")
    ns = (int(n),) * dim if np.isscalar(n) else tuple(int(v) for v in n)
    if len(ns) != dim:
        raise ValueError("one element count per axis")
    shape = tuple(img.shape[::-1])  # W, H(, D)
    means = {"arithmetic": L.ADS_MAP_ARITHMETIC, "geometric": L.ADS_MAP_GEOMETRIC}
    nodes = tuple(v + 1 for v in ns[::-1])
    if out is None:
        out = torch.empty(nodes, dtype=torch.float64, device=img.device)
    elif not (out.is_cuda and out.dtype == torch.float64 and out.is_contiguous() and out.numel() == np.prod(nodes)):
        raise ValueError("out must be a contiguous float64 CUDA tensor of prod(n_a + 1) values")
    stream = C.c_void_p(torch.cuda.current_stream(img.device).cuda_stream)
    pad = [0] * (3 - dim)
    rc = lib.ads_map_from_image(img.data_ptr(), ptype, dim, (C.c_int * 3)(*shape, *pad), int(flip_y),
                                (C.c_int * 3)(*ns, *pad), means[mean], float(scale), float(offset),
                                out.data_ptr(), stream)
    if rc != L.ADS_OK:
        raise L.AdsError(rc, "ads_map_from_image", "")
    return out
