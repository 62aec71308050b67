"""Precision forms: FP32 arithmetic with the populations stored in FP16 or
BF16 as differences from a reference equilibrium, against the FP64 oracle.
Errors are reported per field as relative L2 and L-infinity norms of
(GPU - oracle) over the field scale (the scales of test_gpu_parity)."""
import json
import os

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2002_03644_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELDS = ("rho", "ux", "uy", "theta", "s", "a1")


@pytest.fixture(scope="module")
def hl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2002_03644_gb300 import hlbm
    return hlbm


def errors(got, ref, gamma):
    c = np.sqrt(gamma * ref["theta"] / 3.0).max()
    umax = np.sqrt(ref["ux"] ** 2 + ref["uy"] ** 2).max()
    sc = {"rho": np.abs(ref["rho"]).max(), "ux": umax + c, "uy": umax + c, "theta": ref["theta"].max(),
          "s": np.abs(ref["s"]).max(), "a1": (ref["rho"] * ref["theta"] / 3.0).max()}
    out = {}
    for k in FIELDS:
        d = (got[k] - ref[k]) / sc[k]
        out[k] = {"l2": float(np.sqrt(np.mean(d * d))), "linf": float(np.abs(d).max())}
    return out


# (case, steps, norm asserted).  The smooth vortex is held to L-infinity
# bounds; at the shock tube's discontinuities rounding differences are
# amplified, so L2 is asserted there and L-infinity only reported.
CASES = {
    "vortex256": lambda: (inputs.vortex(n=256, R=8.0), 200, "linf"),
    "sod400": lambda: (inputs.sod(C0=3.875, mu=3e-6, sigma=0.0), 150, "l2"),
}
# bounds per precision over rho, u, theta, s
BOUND = {1: 1e-4, 2: 5e-3, 3: 4e-2}


@pytest.mark.parametrize("case_name", list(CASES))
def test_precision_forms_against_fp64_oracle(hl, case_name):
    case, steps, norm = CASES[case_name]()
    ora = Oracle(case.nx, case.ny, **case.params())
    ora.init(*case.fields())
    ora.step(steps)
    ref = ora.macros()
    report = {}
    for prec, name in ((1, "fp32"), (2, "fp16pop"), (3, "bf16pop")):
        s = hl.Solver(case.nx, case.ny, precision=prec, **case.params())
        s.init(*case.fields())
        s.step(steps)
        got = s.macros()
        s.close()
        e = errors(got, ref, case.gamma)
        report[name] = e
        for k in ("rho", "ux", "uy", "theta", "s"):
            assert np.isfinite(got[k]).all()
            assert e[k][norm] <= BOUND[prec], (name, k, e[k])
    print(f"\nprecision errors {case_name} after {steps} steps:\n" + json.dumps(report, indent=1))
    out = os.environ.get("HLBM_PRECISION_REPORT")
    if out:
        with open(out, "a") as f:
            f.write(json.dumps({"case": case_name, "steps": steps, "errors": report}) + "\n")


def test_precision_forms_four_quadrant_within_the_problems_own_sensitivity(hl):
    """The four-quadrant Riemann problem (96^2, zero-gradient sides) over its
    first 25 steps.  The upwind E1 switches on the sign of round-off
    velocities at the junction, so the result depends on the last bits of
    the data: the oracle fed the initial fields rounded to FP32 ends, in L2
    over the field scales, about 4e-4 (rho) away from the oracle fed them in
    FP64.  No form that stores FP32 or less can do better, so each form's L2
    error is held to the larger of its bound and 3x that measured
    sensitivity, field by field, and reported."""
    case, steps = inputs.four_quadrant(n=96), 25
    ora = Oracle(case.nx, case.ny, **case.params())
    ora.init(*case.fields())
    ora.step(steps)
    ref = ora.macros()
    o32 = Oracle(case.nx, case.ny, **case.params())
    o32.init(*[np.asarray(x).astype(np.float32).astype(np.float64) for x in case.fields()])
    o32.step(steps)
    sens = errors(o32.macros(), ref, case.gamma)
    report = {"oracle_fp32_inputs": sens}
    for prec, name in ((1, "fp32"), (2, "fp16pop"), (3, "bf16pop")):
        s = hl.Solver(case.nx, case.ny, precision=prec, **case.params())
        s.init(*case.fields())
        s.step(steps)
        got = s.macros()
        s.close()
        e = errors(got, ref, case.gamma)
        report[name] = e
        for k in ("rho", "ux", "uy", "theta", "s"):
            assert np.isfinite(got[k]).all()
            assert e[k]["l2"] <= max(BOUND[prec], 3.0 * sens[k]["l2"]), (name, k, e[k], sens[k])
    print(f"\nprecision errors quadrant96 after {steps} steps:\n" + json.dumps(report, indent=1))
    out = os.environ.get("HLBM_PRECISION_REPORT")
    if out:
        with open(out, "a") as f:
            f.write(json.dumps({"case": "quadrant96", "steps": steps, "errors": report}) + "\n")


def test_four_quadrant_full_size_first_step(hl):
    """The four-quadrant Riemann problem at its full 4096^2 size (zero-gradient
    sides: the marching kernel's general form), one step, every cell: FP32
    within 1e-4 and the 16-bit storage forms within their bounds, in
    L-infinity.  After one step no velocity is yet round-off at the junction
    (the oracle moved by 2^-50 stays within 1e-15 of itself), so the
    pointwise bounds hold on this discontinuous data."""
    from oracle.oracle import max_threads
    case = inputs.four_quadrant(n=4096)
    ora = Oracle(case.nx, case.ny, **case.params())
    ora.set_threads(max_threads())
    ora.init(*case.fields())
    ora.step(1)
    ref = ora.macros()
    del ora
    report = {}
    for prec, name in ((1, "fp32"), (2, "fp16pop"), (3, "bf16pop")):
        s = hl.Solver(case.nx, case.ny, precision=prec, **case.params())
        s.init(*case.fields())
        s.step(1)
        got = s.macros()
        s.close()
        e = errors(got, ref, case.gamma)
        report[name] = {k: e[k]["linf"] for k in FIELDS}
        for k in ("rho", "ux", "uy", "theta", "s"):
            assert np.isfinite(got[k]).all()
            assert e[k]["linf"] <= BOUND[prec], (name, k, e[k])
    print("\nfour-quadrant 4096^2, one step, L-infinity: " + json.dumps(report))


def _report(name, steps, report):
    print(f"\nprecision errors {name} after {steps} steps:\n" + json.dumps(report, indent=1))
    out = os.environ.get("HLBM_PRECISION_REPORT")
    if out:
        with open(out, "a") as f:
            f.write(json.dumps({"case": name, "steps": steps, "errors": report}) + "\n")


def test_precision_forms_four_quadrant_512_on_the_longest_running_setting(hl):
    """The four-quadrant configuration's 512^2 error run, on the setting of
    the paper's own knobs that runs longest before the scheme leaves its range
    of stability (finite-difference Phi, sigma = 0.1, C_0 = 10, mu = 0.01: 670
    of the 1536 steps to t = 0.3 in the oracle), over its first 100 steps.
    The problem is chaotic under round-off: the oracle fed one quadrant's
    density larger by one part in 2^50 departs from itself by L2 about 2e-4
    of the density scale.  FP32 and the moment state are held to 3x that
    measured sensitivity, the 16-bit forms to their L2 bounds, field by
    field; all are reported."""
    from oracle.oracle import max_threads
    n, steps = 512, 100
    case = inputs.four_quadrant(n=n, C0=10.0, mu=0.01, sigma=0.1)
    case.phi_mode = 1

    def oracle(rho):
        o = Oracle(case.nx, case.ny, **case.params())
        o.set_threads(max_threads())
        o.init(rho, case.ux, case.uy, case.theta)
        o.step(steps)
        return o.macros()
    ref = oracle(case.rho)
    r2 = case.rho.copy()
    r2[n // 2:, n // 2:] *= 1.0 + 2.0 ** -50
    sens = errors(oracle(r2), ref, case.gamma)
    report = {"oracle_2^-50": sens}
    for prec, name in ((1, "fp32"), (4, "moments"), (2, "fp16pop"), (3, "bf16pop")):
        s = hl.Solver(case.nx, case.ny, precision=prec, **case.params())
        s.init(*case.fields())
        s.step(steps)
        got = s.macros()
        s.close()
        e = errors(got, ref, case.gamma)
        report[name] = e
        for k in ("rho", "ux", "uy", "theta", "s"):
            assert np.isfinite(got[k]).all()
            bound = 3.0 * sens[k]["l2"] if prec in (1, 4) else BOUND[prec]
            assert e[k]["l2"] <= bound, (name, k, e[k], sens[k])
    _report("quadrant512", steps, report)


def test_16bit_error_follows_the_departure_from_the_reference(hl):
    """Why FP16 storage misses 1e-4 on the configured vortex: it stores
    F_i - f_ref_i with 11 significant bits and one reference equilibrium per
    case, so its error follows the size of that difference, i.e. the flow's
    departure from the mean state.  On the 256^2 vortex (R = 8, 200 steps)
    halving and quartering the vortex strength shrinks the FP16 error of rho
    by more than 2x in all, to within 1e-4 at a quarter of the strength."""
    rep = {}
    for beta in (0.2, 0.1, 0.05):
        case = inputs.vortex(n=256, R=8.0, beta=beta)
        ora = Oracle(case.nx, case.ny, **case.params())
        ora.init(*case.fields())
        ora.step(200)
        ref = ora.macros()
        s = hl.Solver(case.nx, case.ny, precision=2, **case.params())
        s.init(*case.fields())
        s.step(200)
        rep[beta] = errors(s.macros(), ref, case.gamma)
        s.close()
    e = [rep[b]["rho"]["linf"] for b in (0.2, 0.1, 0.05)]
    assert e[0] > e[1] > e[2] and e[0] > 2.0 * e[2], e
    assert e[2] <= 1e-4, e
    _report("vortex256_fp16_by_strength", 200, {f"beta={b}": rep[b] for b in rep})


@pytest.mark.parametrize("prec", [2, 3])
def test_16bit_checkpoint_keeps_the_reference(hl, prec):
    case = inputs.vortex(n=96, R=6.0)
    a = hl.Solver(case.nx, case.ny, precision=prec, **case.params())
    a.init(*case.fields())
    a.step(5)
    blob = a.state()
    a.step(5)
    b = hl.Solver(case.nx, case.ny, precision=prec, **case.params())
    b.set_state(blob)
    b.step(5)
    ma, mb = a.macros(), b.macros()
    for k in ma:
        assert np.array_equal(ma[k], mb[k]), k
