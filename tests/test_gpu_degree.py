"""The saturation step for B-splines of degree 2, 3 and 4 (ads_degree_*)
against the FP64 oracle of the same degree, through the C ABI.

The oracle's degree-p path is pinned on the CPU (test_oracle_pins.py: mass
matrix, partition of unity, the Kronecker solve against a dense one).  Here
the GPU step must agree with it to FP64 rounding on meshes that are small,
ragged and larger than one block of threads, with a porosity map, gravity and
injectors as well as producers; at degree 2 it must also agree with the
quadratic context path (ads_saturation_step).
"""
import ctypes as C

import numpy as np
import pytest

from oracle.ads import AdsOracle

pytestmark = pytest.mark.gpu


def _case(n, p, seed):
    from paper_2604_20731_gb300 import scenario as scn
    sc = scn.make_scenario(2, n, seed=seed, S0="random", grav=0.4)
    sc.sources = [
        scn.Source(center=(0.2, 0.3), rate=1.3, kind=scn.SRC_INJECT),
        scn.Source(center=(0.7, 0.25), rate=0.6, sigma=0.05, kind=scn.SRC_INJECT),
        scn.Source(center=(0.8, 0.8), rate=1.1, kind=scn.SRC_PRODUCE),
    ]
    rng = np.random.default_rng(seed + 1)
    sc.phi_map = 0.1 + 0.3 * rng.uniform(size=(n + 1, n + 1))
    sc.p = p
    nb = n + p
    S = rng.uniform(-0.1, 1.1, size=(nb, nb))
    P = rng.normal(size=(nb, nb))
    return sc, S, P


def _plan(lib, sc, p):
    from paper_2604_20731_gb300.solver import make_params
    params = make_params(sc, "f64", any_degree=True)
    plan = C.c_void_p()
    rc = lib.ads_degree_plan_create(C.byref(params), p, C.byref(plan))
    assert rc == 0 and plan.value
    return plan, params


@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("n", [4, 33, 160])
def test_degree_step_matches_oracle(p, n):
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g
    g.build()
    from paper_2604_20731_gb300 import _lib
    lib = _lib.load()
    sc, S, P = _case(n, p, seed=100 + 7 * n + p)
    plan, _ = _plan(lib, sc, p)
    try:
        assert lib.ads_degree_coeffs(plan) == n + p
        dev = torch.device("cuda", 0)
        K = torch.from_numpy(np.ascontiguousarray(sc.K, dtype=np.float64)).to(dev)
        phi = torch.from_numpy(np.ascontiguousarray(sc.phi_map)).to(dev)
        Sd = torch.from_numpy(S).to(dev)
        Pd = torch.from_numpy(P).to(dev)
        out = torch.empty_like(Sd)
        out2 = torch.empty_like(Sd)
        dt = 2e-4
        st = torch.cuda.Stream(device=dev)
        h = C.c_void_p(st.cuda_stream)
        torch.cuda.synchronize()
        # two steps: S1 = step(S), S2 = step(S1)
        assert lib.ads_degree_step(plan, K.data_ptr(), phi.data_ptr(), Sd.data_ptr(), Pd.data_ptr(), dt,
                                   out.data_ptr(), h) == 0
        assert lib.ads_degree_step(plan, K.data_ptr(), phi.data_ptr(), out.data_ptr(), Pd.data_ptr(), dt,
                                   out2.data_ptr(), h) == 0
        mass = C.c_double()
        assert lib.ads_degree_mass(plan, out2.data_ptr(), C.byref(mass), h) == 0
        a = AdsOracle(sc)
        ref1 = a.step(S, P, dt)
        ref2 = a.step(ref1, P, dt)
        for got, ref in ((out.cpu().numpy(), ref1), (out2.cpu().numpy(), ref2)):
            assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
        assert mass.value == pytest.approx(a.mesh.integral(ref2), rel=1e-12, abs=1e-14)
        # the step conserves mass up to the sources: int S1 - int S - dt int q_g / phi = 0
        m0 = C.c_double()
        assert lib.ads_degree_mass(plan, Sd.data_ptr(), C.byref(m0), h) == 0
        m1 = C.c_double()
        assert lib.ads_degree_mass(plan, out.data_ptr(), C.byref(m1), h) == 0
        assert m1.value - m0.value == pytest.approx(a.source_integral(S, dt), rel=1e-9, abs=1e-15)
        # without a porosity map: params.phi everywhere
        sc.phi_map = None
        assert lib.ads_degree_step(plan, K.data_ptr(), None, Sd.data_ptr(), Pd.data_ptr(), dt,
                                   out.data_ptr(), h) == 0
        st.synchronize()
        ref = AdsOracle(sc).step(S, P, dt)
        assert np.abs(out.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    finally:
        lib.ads_degree_plan_destroy(plan)


def test_degree_two_matches_the_quadratic_context_path():
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g
    g.build()
    from paper_2604_20731_gb300 import _lib
    from paper_2604_20731_gb300.solver import HybridSolver
    lib = _lib.load()
    n = 77
    sc, S, P = _case(n, 2, seed=5)
    s = HybridSolver(sc, width=None, ads_dtype="f64")
    plan, _ = _plan(lib, sc, 2)
    try:
        s.set_saturation(S)
        s.set_pressure(P)
        dt = 3e-4
        s.saturation_step(dt, 1)
        ref = s.get("S")
        dev = torch.device("cuda", 0)
        K = torch.from_numpy(np.ascontiguousarray(sc.K, dtype=np.float64)).to(dev)
        phi = torch.from_numpy(np.ascontiguousarray(sc.phi_map)).to(dev)
        Sd, Pd = torch.from_numpy(S).to(dev), torch.from_numpy(P).to(dev)
        out = torch.empty_like(Sd)
        torch.cuda.synchronize()
        assert lib.ads_degree_step(plan, K.data_ptr(), phi.data_ptr(), Sd.data_ptr(), Pd.data_ptr(), dt,
                                   out.data_ptr(), None) == 0
        torch.cuda.synchronize()
        assert np.abs(out.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    finally:
        lib.ads_degree_plan_destroy(plan)
        s.close()


def test_degree_step_refuses_aliasing_and_bad_steps():
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g
    g.build()
    from paper_2604_20731_gb300 import _lib
    lib = _lib.load()
    sc, S, P = _case(8, 3, seed=9)
    plan, _ = _plan(lib, sc, 3)
    try:
        dev = torch.device("cuda", 0)
        K = torch.from_numpy(np.ascontiguousarray(sc.K, dtype=np.float64)).to(dev)
        Sd, Pd = torch.from_numpy(S).to(dev), torch.from_numpy(P).to(dev)
        out = torch.empty_like(Sd)
        for dt in (0.0, -1.0, float("inf"), float("nan")):
            assert lib.ads_degree_step(plan, K.data_ptr(), None, Sd.data_ptr(), Pd.data_ptr(), dt,
                                       out.data_ptr(), None) == 1
        assert lib.ads_degree_step(plan, K.data_ptr(), None, Sd.data_ptr(), Pd.data_ptr(), 1e-4,
                                   Sd.data_ptr(), None) == 1
        assert lib.ads_degree_step(plan, K.data_ptr(), None, Sd.data_ptr(), Pd.data_ptr(), 1e-4,
                                   Pd.data_ptr(), None) == 1
        assert lib.ads_degree_step(plan, None, None, Sd.data_ptr(), Pd.data_ptr(), 1e-4,
                                   out.data_ptr(), None) == 1
    finally:
        lib.ads_degree_plan_destroy(plan)


@pytest.mark.parametrize("p,n", [(2, 6), (3, 5), (4, 7)])
def test_degree_step_vjp_matches_oracle_finite_differences(p, n):
    """ads_degree_step_vjp against central differences of the oracle's step:
    J = lambda . step(S, P, sources), along random directions in S and P and
    along each source's rate and centre.  S stays inside (0, 1) at the Gauss
    points, where the mobility is smooth."""
    import dataclasses
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g
    g.build()
    from paper_2604_20731_gb300 import _lib
    lib = _lib.load()
    sc, _, P = _case(n, p, seed=300 + n + p)
    nb = n + p
    rng = np.random.default_rng(40 + p)
    S = rng.uniform(0.3, 0.7, size=(nb, nb))
    lam = rng.normal(size=(nb, nb))
    dt = 5e-3
    plan, _ = _plan(lib, sc, p)
    try:
        dev = torch.device("cuda", 0)
        t = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(dev)
        K, phi, Sd, Pd, Ld = t(sc.K), t(sc.phi_map), t(S), t(P), t(lam)
        gS, gP = torch.empty_like(Sd), torch.empty_like(Sd)
        gsrc = (C.c_double * (3 * len(sc.sources)))()
        torch.cuda.synchronize()
        assert lib.ads_degree_step_vjp(plan, K.data_ptr(), phi.data_ptr(), Sd.data_ptr(), Pd.data_ptr(), dt,
                                       Ld.data_ptr(), gS.data_ptr(), gP.data_ptr(), gsrc, None) == 0
        torch.cuda.synchronize()
        gS, gP, gsrc = gS.cpu().numpy(), gP.cpu().numpy(), np.array(gsrc[:])
    finally:
        lib.ads_degree_plan_destroy(plan)

    def J(S_, P_, sources=None):
        sc2 = dataclasses.replace(sc, sources=sources if sources is not None else sc.sources)
        sc2.p = p
        return float(np.sum(lam * AdsOracle(sc2).step(S_, P_, dt)))

    # central differences with one Richardson step: (4 D(e/2) - D(e)) / 3
    # cancels the e^2 term (the Gaussians of width 0.03 on a coarse mesh make
    # J vary quickly with a source's centre)
    eps = 1e-4

    def rich(f):
        d1 = (f(eps) - f(-eps)) / (2 * eps)
        d2 = (f(eps / 2) - f(-eps / 2)) / eps
        return (4 * d2 - d1) / 3

    for _ in range(2):
        dS, dP = rng.normal(size=(nb, nb)), rng.normal(size=(nb, nb))
        fd_S = rich(lambda e: J(S + e * dS, P))
        fd_P = rich(lambda e: J(S, P + e * dP))
        assert np.sum(gS * dS) == pytest.approx(fd_S, rel=1e-6, abs=1e-9)
        assert np.sum(gP * dP) == pytest.approx(fd_P, rel=1e-6, abs=1e-9)
    for k, src in enumerate(sc.sources):
        for j, field in enumerate(("rate", "cx", "cy")):
            def moved(d):
                out = list(sc.sources)
                if field == "rate":
                    out[k] = dataclasses.replace(src, rate=src.rate + d)
                else:
                    c = list(src.center)
                    c[0 if field == "cx" else 1] += d
                    out[k] = dataclasses.replace(src, center=tuple(c))
                return out
            fd = rich(lambda e: J(S, P, moved(e)))
            assert gsrc[3 * k + j] == pytest.approx(fd, rel=1e-6, abs=1e-9), (k, field)


@pytest.mark.parametrize("p,n", [(2, 20), (3, 33), (4, 17)])
def test_degree_projection_and_step_size_match_oracle(p, n):
    """The projection of nodal values into the degree-p splines and the CFL
    step size against the oracle (project_nodal, AdsOracle.cfl_dt)."""
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g
    g.build()
    from oracle.hybrid import project_nodal
    from paper_2604_20731_gb300 import _lib
    lib = _lib.load()
    sc, _, P = _case(n, p, seed=500 + n + p)
    rng = np.random.default_rng(n)
    nodal = rng.normal(size=(n + 1, n + 1))
    nodal[0, :] = nodal[-1, :] = nodal[:, 0] = nodal[:, -1] = 0.0
    plan, _ = _plan(lib, sc, p)
    try:
        dev = torch.device("cuda", 0)
        t = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(dev)
        K, phi, Pd, Nd = t(sc.K), t(sc.phi_map), t(P), t(nodal)
        out = torch.empty((n + p, n + p), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        assert lib.ads_degree_project(plan, Nd.data_ptr(), out.data_ptr(), None) == 0
        dt = C.c_double()
        assert lib.ads_degree_cfl_dt(plan, K.data_ptr(), phi.data_ptr(), Pd.data_ptr(), 0.1, 0.05,
                                     float("inf"), C.byref(dt), None) == 0
        torch.cuda.synchronize()
        a = AdsOracle(sc)
        ref = project_nodal(a.mesh, nodal)
        assert np.abs(out.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
        assert dt.value == pytest.approx(a.cfl_dt(P, cfl=0.1, src_frac=0.05), rel=1e-12)
        dt2 = C.c_double()
        assert lib.ads_degree_cfl_dt(plan, K.data_ptr(), phi.data_ptr(), Pd.data_ptr(), 0.1, 0.05,
                                     1e-9, C.byref(dt2), None) == 0
        assert dt2.value == 1e-9
        for bad in ((0.0, 0.05), (0.1, -1.0), (float("nan"), 0.05)):
            assert lib.ads_degree_cfl_dt(plan, K.data_ptr(), None, Pd.data_ptr(), bad[0], bad[1], 1.0,
                                         C.byref(dt2), None) == 1
    finally:
        lib.ads_degree_plan_destroy(plan)


def test_gradient_through_several_steps_for_well_placement():
    """DegreePlan.steps_with_gradient chains the vector-Jacobian products
    backward through three explicit steps (degree 3): the gradient of
    J = lambda . S_3 with respect to S_0, P and each source's rate and centre
    against Richardson-extrapolated central differences of three oracle
    steps."""
    import dataclasses
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g
    g.build()
    from paper_2604_20731_gb300.solver import DegreePlan
    p, n, steps, dt = 3, 6, 3, 4e-3
    sc, _, P = _case(n, p, seed=77)
    nb = n + p
    rng = np.random.default_rng(78)
    S0 = rng.uniform(0.3, 0.7, size=(nb, nb))
    lam = rng.normal(size=(nb, nb))
    plan = DegreePlan(sc, p)
    try:
        dev = torch.device("cuda", 0)
        t = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(dev)
        K, phi = t(sc.K), t(sc.phi_map)
        Sn, gS0, gP, gsrc = plan.steps_with_gradient(K, phi, t(S0), t(P), dt, steps, t(lam))
        torch.cuda.synchronize()
        Sn, gS0, gP = Sn.cpu().numpy(), gS0.cpu().numpy(), gP.cpu().numpy()
    finally:
        plan.close()

    def run(S_, P_, sources=None):
        sc2 = dataclasses.replace(sc, sources=sources if sources is not None else sc.sources)
        sc2.p = p
        a = AdsOracle(sc2)
        for _ in range(steps):
            S_ = a.step(S_, P_, dt)
        return S_

    ref = run(S0, P)
    assert np.abs(Sn - ref).max() <= 1e-12 * np.abs(ref).max()
    J = lambda *args: float(np.sum(lam * run(*args)))
    eps = 1e-4

    def rich(f):
        d1 = (f(eps) - f(-eps)) / (2 * eps)
        d2 = (f(eps / 2) - f(-eps / 2)) / eps
        return (4 * d2 - d1) / 3

    dS, dP = rng.normal(size=(nb, nb)), rng.normal(size=(nb, nb))
    assert np.sum(gS0 * dS) == pytest.approx(rich(lambda e: J(S0 + e * dS, P)), rel=1e-6, abs=1e-9)
    assert np.sum(gP * dP) == pytest.approx(rich(lambda e: J(S0, P + e * dP)), rel=1e-6, abs=1e-9)
    for k, src in enumerate(sc.sources):
        for j, field in enumerate(("rate", "cx", "cy")):
            def moved(d):
                out = list(sc.sources)
                if field == "rate":
                    out[k] = dataclasses.replace(src, rate=src.rate + d)
                else:
                    c = list(src.center)
                    c[0 if field == "cx" else 1] += d
                    out[k] = dataclasses.replace(src, center=tuple(c))
                return out
            fd = rich(lambda e: J(S0, P, moved(e)))
            assert gsrc[k, j] == pytest.approx(fd, rel=1e-6, abs=1e-9), (k, field)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_projection_adjoint_dot_product(p):
    """ads_degree_project_vjp is the adjoint of ads_degree_project (itself
    pinned to the oracle's projection): g . project(u) = project_vjp(g) . u
    for random u and g, on a ragged mesh."""
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g_
    g_.build()
    from paper_2604_20731_gb300.solver import DegreePlan
    n = 37
    sc, _, _ = _case(n, p, seed=300 + p)
    rng = np.random.default_rng(301 + p)
    u = rng.normal(size=(n + 1, n + 1))
    g = rng.normal(size=(n + p, n + p))
    plan = DegreePlan(sc, p)
    try:
        dev = torch.device("cuda", 0)
        ud, gd = torch.from_numpy(u).to(dev), torch.from_numpy(g).to(dev)
        P, gu = torch.empty_like(gd), torch.empty_like(ud)
        plan.project(ud, P)
        plan.project_vjp(gd, gu)
        torch.cuda.synchronize()
        lhs = float(np.sum(g * P.cpu().numpy()))
        rhs = float(np.sum(gu.cpu().numpy() * u))
    finally:
        plan.close()
    assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-14)


@pytest.mark.parametrize("p", [2, 3])
def test_gradient_with_respect_to_the_network_parameters(p):
    """pressure_network_gradient: J = lambda . S_n after two steps whose
    pressure is the FP64 network's nodal values projected into the degree-p
    splines.  The gradient with respect to theta (through the steps, the
    projection and the network's hand-written backward) against
    Richardson-extrapolated central differences of the oracle's J(theta):
    its network, projection and steps."""
    import dataclasses
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g_
    g_.build()
    from oracle.hybrid import HybridOracle
    from paper_2604_20731_gb300 import scenario as scn
    from paper_2604_20731_gb300.solver import DegreePlan, HybridSolver, pressure_network_gradient
    n, steps, dt, width = 8, 2, 2e-3, 64
    sc = scn.make_scenario(2, n, seed=410 + p, S0="random", grav=0.3)
    theta = scn.make_theta0(2, width, 4, seed=411 + p)
    rng = np.random.default_rng(412 + p)
    nb = n + p
    S0 = rng.uniform(0.2, 0.8, size=(nb, nb))
    lam = rng.normal(size=(nb, nb))
    solver = HybridSolver(sc, width=width, crv_dtype="f64", ads_dtype="f64")
    scp = dataclasses.replace(sc)
    scp.p = p
    plan = DegreePlan(scp, p)
    try:
        solver.set_theta(theta)
        dev = torch.device("cuda", 0)
        t = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(dev)
        Sn, gS0, gth, gsrc = pressure_network_gradient(solver, plan, t(sc.K), None, t(S0), dt, steps, t(lam))
        torch.cuda.synchronize()
        Sn = Sn.cpu().numpy()
    finally:
        plan.close()
        solver.close()
    ho = HybridOracle(scp, width)

    def run(th):
        P = ho.project(th)
        S = S0
        for _ in range(steps):
            S = ho.ads.step(S, P, dt)
        return S

    ref = run(theta)
    assert np.abs(Sn - ref).max() <= 1e-12 * np.abs(ref).max()
    J = lambda th: float(np.sum(lam * run(th)))
    eps = 1e-4
    for k in range(3):
        d = rng.normal(size=theta.shape)
        d /= np.linalg.norm(d)
        f = lambda e: J(theta + e * d)
        d1 = (f(eps) - f(-eps)) / (2 * eps)
        d2 = (f(eps / 2) - f(-eps / 2)) / eps
        fd = (4 * d2 - d1) / 3
        assert float(np.dot(gth, d)) == pytest.approx(fd, rel=1e-6, abs=1e-10), k
