"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake (a wrong index, a transposed operand, a dropped
or sign-flipped term, a wrong coefficient) into a copy of the oracle's C
source, builds it with gcc, points the oracle module at the mutant and runs
the pin tests; at least one pin must fail.  Mistakes are planted in the CPU
oracle only.
"""
import ctypes
import inspect
import os
import subprocess

import pytest

import oracle
import test_oracle_adjoint_pins as adj_pins
import test_oracle_pins as fwd_pins

MUTATIONS = {
    "su_x_wrong_index": ("- u[AT(ip, j, k)] * (u[AT(i, j, k)] + u[AT(ip, j, k)]));",
                         "- u[AT(ip, j, k)] * (u[AT(i, j, k)] + u[AT(im, j, k)]));"),
    "su_y_average_wrong_column": ("(v[AT(i, jm, k)] + v[AT(ip, jm, k)])",
                                  "(v[AT(i, jm, k)] + v[AT(im, jm, k)])"),
    "su_y_sign_flip": ("su = su + tcy * (u[AT(i, jm, k)]", "su = su - tcy * (u[AT(i, jm, k)]"),
    "su_vertical_coeffs_swapped": (
        "su = su + tzc1[k] * u[AT(i, j, k - 1)] * (w[AT(i, j, k - 1)] + w[AT(ip, j, k - 1)])\n"
        "                    - tzc2[k]",
        "su = su + tzc2[k] * u[AT(i, j, k - 1)] * (w[AT(i, j, k - 1)] + w[AT(ip, j, k - 1)])\n"
        "                    - tzc1[k]"),
    "sv_x_transposed_operand": ("(u[AT(im, j, k)] + u[AT(im, jp, k)])",
                                "(u[AT(im, j, k)] + u[AT(ip, jp, k)])"),
    "sv_lower_flux_dropped": (
        "sv = sv + tzc1[k] * v[AT(i, j, k - 1)] * (w[AT(i, j, k - 1)] + w[AT(i, jp, k - 1)])\n"
        "                    - tzc2[k]",
        "sv = sv + 0.0 * v[AT(i, j, k - 1)] * (w[AT(i, j, k - 1)] + w[AT(i, jp, k - 1)])\n"
        "                    - tzc2[k]"),
    "sw_upper_uses_tzd1": ("- tzd2[k] * w[AT(i, j, k + 1)]", "- tzd1[k] * w[AT(i, j, k + 1)]"),
    "sw_x_average_wrong_level": ("(u[AT(i, j, k)] + u[AT(i, j, k + 1)]));",
                                 "(u[AT(i, j, k)] + u[AT(i, j, k - 1)]));"),
    "tcx_half_width": ("tcxy[0] = 1.0 / (4.0 * dx);", "tcxy[0] = 1.0 / (2.0 * dx);"),
    "tzc1_density_level": ("tzc1[k] = rho[k - 1] /", "tzc1[k] = rhon[k - 1] /"),
    "tzd_uses_w_spacing": ("double dznk1 = zn[k + 1] - zn[k];", "double dznk1 = z[k + 1] - z[k];"),
    "adjoint_product_rule_operand": ("gc[cc] += s * fa[a];", "gc[cc] += s * fb[b];"),
    "adjoint_cotangent_index": ("l = dsv[q]; /* sv terms */", "l = dsu[q]; /* sv terms */"),
    "sv_y_upper_sign_flip": ("- v[AT(i, jp, k)] * (v[AT(i, j, k)] + v[AT(i, jp, k)]));",
                             "+ v[AT(i, jp, k)] * (v[AT(i, j, k)] + v[AT(i, jp, k)]));"),
    "sv_upper_vertical_wrong_column": (
        "- tzc2[k] * v[AT(i, j, k + 1)] * (w[AT(i, j, k)] + w[AT(i, jp, k)]);",
        "- tzc2[k] * v[AT(i, j, k + 1)] * (w[AT(i, j, k)] + w[AT(i, j, k)]);"),
    "sw_x_lower_wrong_level": ("sw = tcx * (w[AT(im, j, k)] * (u[AT(im, j, k)] + u[AT(im, j, k + 1)])",
                               "sw = tcx * (w[AT(im, j, k)] * (u[AT(im, j, k)] + u[AT(im, j, k - 1)])"),
    "sw_y_upper_wrong_row": ("- w[AT(i, jp, k)] * (v[AT(i, j, k)] + v[AT(i, j, k + 1)]));",
                             "- w[AT(i, jp, k)] * (v[AT(i, jp, k)] + v[AT(i, j, k + 1)]));"),
    "sw_lower_vertical_wrong_operand": ("sw = sw + tzd1[k] * w[AT(i, j, k - 1)] *",
                                        "sw = sw + tzd1[k] * w[AT(i, j, k)] *"),
    "tzd2_density_level": ("tzd2[k] = rhon[k + 1] /", "tzd2[k] = rhon[k] /"),
    "tzc2_density": ("tzc2[k] = rho[k] / (4.0 * dzk * rhon[k]);",
                     "tzc2[k] = rhon[k] / (4.0 * dzk * rhon[k]);"),
    "adjoint_su_y_target_swapped": (
        "term(tcy, l, u, AT(i, jm, k), v, AT(i, jm, k), v, AT(ip, jm, k), du, dv, dv);",
        "term(tcy, l, u, AT(i, jm, k), v, AT(i, jm, k), v, AT(ip, jm, k), du, dv, du);"),
    "adjoint_sw_vertical_coefficient": ("term(tzd1[k], l, w, AT(i, j, k - 1)",
                                        "term(tzd2[k], l, w, AT(i, j, k - 1)"),
    "adjoint_sv_x_index": (
        "term(-tcx, l, v, AT(ip, j, k), u, AT(i, j, k), u, AT(i, jp, k), dv, du, du);",
        "term(-tcx, l, v, AT(ip, j, k), u, AT(i, j, k), u, AT(ip, jp, k), dv, du, du);"),
}


def _pins():
    out = []
    for mod in (fwd_pins, adj_pins):
        for name, fn in inspect.getmembers(mod, inspect.isfunction):
            if not name.startswith("test_"):
                continue
            marks = getattr(fn, "pytestmark", [])
            params = [m for m in marks if m.name == "parametrize"]
            if params:
                argnames = [a.strip() for a in params[0].args[0].split(",")]
                for vals in params[0].args[1]:
                    out.append((f"{name}{vals}", fn, dict(zip(argnames, vals))))
            else:
                out.append((name, fn, {}))
    return out


@pytest.fixture(scope="module")
def source():
    with open(oracle._SRC) as f:
        return f.read()


@pytest.mark.parametrize("mutation", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(mutation, source, tmp_path):
    old, new = MUTATIONS[mutation]
    assert source.count(old) == 1, f"mutation anchor not unique: {mutation}"
    src = tmp_path / "mutant.c"
    src.write_text(source.replace(old, new))
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", *oracle.CFLAGS, "-o", str(so), str(src)], check=True)
    saved = dict(oracle._lib_handles)
    oracle._lib_handles.clear()
    real_build = oracle.build
    oracle.build = lambda force=False, openmp=False: str(so)
    caught = []
    try:
        for name, fn, kwargs in _pins():
            try:
                fn(**kwargs)
            except AssertionError:
                caught.append(name)
    finally:
        oracle.build = real_build
        oracle._lib_handles.clear()
        oracle._lib_handles.update(saved)
    assert caught, f"no pin caught mutation {mutation}"


# Mistakes planted into the (Python) integration step of the oracle.
INTEGRATE_MUTATIONS = {
    "integrate_sign_flip": ("bf + dt * s for bf", "bf - dt * s for bf"),
    "integrate_step_dropped": ("bf + dt * s for bf", "bf + s for bf"),
    "integrate_half_step": ("bf + dt * s for bf", "bf + 0.5 * dt * s for bf"),
    "integrate_ignores_base": ("base = (u, v, w)\n    b = [_f64(x) for x in base]",
                               "base = (u, v, w)\n    b = [_f64(x) for x in (u, v, w)]"),
    "integrate_fields_rotated": ("zip(b, (su, sv, sw))", "zip(b, (sv, sw, su))"),
}


@pytest.mark.parametrize("mutation", sorted(INTEGRATE_MUTATIONS))
def test_integrate_pins_catch_planted_mistake(mutation):
    import test_oracle_integrate_pins as int_pins
    old, new = INTEGRATE_MUTATIONS[mutation]
    src = inspect.getsource(oracle.integrate)
    assert src.count(old) == 1, f"mutation anchor not unique: {mutation}"
    ns = dict(vars(oracle))
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    real = oracle.integrate
    oracle.integrate = ns["integrate"]
    caught = []
    try:
        for name, fn in inspect.getmembers(int_pins, inspect.isfunction):
            if not name.startswith("test_"):
                continue
            params = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
            cases = [{}]
            if params:
                argnames = [a.strip() for a in params[0].args[0].split(",")]
                cases = [dict(zip(argnames, vals if isinstance(vals, tuple) else (vals,)))
                         for vals in params[0].args[1]]
            for kw in cases:
                try:
                    fn(**kw)
                except (AssertionError, pytest.fail.Exception):
                    caught.append(name)
    finally:
        oracle.integrate = real
    assert caught, f"no pin caught mutation {mutation}"
