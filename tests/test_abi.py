"""The C-ABI library builds, loads, exports every symbol include/vp.h
declares, and carries quadrature tables bit-identical to the oracle's
independently generated ones.  No GPU needed."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = ""
    for name in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if name.endswith(".h"):
            src += open(os.path.join(ROOT, "include", name)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vp_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2205_04401_gb300 import vp
    return vp.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["vp_mesh_upload", "vp_nearfield_build", "vp_potential_eval", "vp_potential_eval_batch"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    assert lib.vp_status_str(0) == b"VP_OK"
    assert lib.vp_status_str(-7) == b"VP_ERR_NO_DEVICE"
    assert lib.vp_status_str(5) == b"VP_UNKNOWN"


@pytest.mark.parametrize("which,name", [(16, "far16"), (19, "far19"), (33, "near33")])
def test_tables_match_oracle_bitwise(tables, which, name):
    from paper_2205_04401_gb300 import vp
    x, y, w, what = vp.rule_table(which)
    r = tables[name]
    assert np.array_equal(x, r["x"]) and np.array_equal(y, r["y"]) and np.array_equal(w, r["w"])
    assert what == r["what"]


def test_radial_rule_of_the_self_weights():
    """The library's 5-point radial rule (float-float self weights) on the
    Gauss-Legendre nodes of [0, 1]: sum_i w_i r_i^k = int_0^1 r r^k dr =
    1/(k+2) and sum_i y_i r_i^k = int_0^1 r r^k log r dr = -1/(k+2)^2 for
    k <= 4, the radial integrands of the P_4 moments (Section 3.4), checked
    in exact rational arithmetic on the stored doubles; the log weights are
    not exact at k = 5 (five nodes fix five moments)."""
    from fractions import Fraction
    from paper_2205_04401_gb300 import vp
    r, y, w, _ = vp.rule_table(5)
    assert len(r) == 5 and np.all((r > 0) & (r < 1)) and np.all(np.diff(r) > 0)
    R, Wa, Wb = ([Fraction(v) for v in a] for a in (r, w, y))
    for k in range(5):
        sa = sum(a * x ** k for a, x in zip(Wa, R))
        sb = sum(b * x ** k for b, x in zip(Wb, R))
        assert abs(float(sa - Fraction(1, k + 2))) < 4e-16
        assert abs(float(sb + Fraction(1, (k + 2) ** 2))) < 4e-16
    sb5 = sum(b * x ** 5 for b, x in zip(Wb, R))
    assert abs(float(sb5 + Fraction(1, 49))) > 1e-10


def test_1d_tables_match_oracle_bitwise(tables):
    from paper_2205_04401_gb300 import vp
    x, _, w, _ = vp.rule_table(8)
    assert np.array_equal(x, tables["ggq8"]["r"]) and np.array_equal(w, tables["ggq8"]["w"])
    x, _, w, _ = vp.rule_table(116)
    assert np.array_equal(x, tables["gl16"]["x"]) and np.array_equal(w, tables["gl16"]["w"])


def test_bad_arguments_return_codes(lib):
    # invalid handles and arguments are reported, never crash
    assert lib.vp_potential_eval(None, None, None, 1, None, 0, None) == -8
    assert lib.vp_mesh_upload(None, None, 0, None, 0, 19, None, None) == -8
    h = C.c_void_p()
    rc = lib.vp_create(C.byref(h), 10_000)
    assert rc == -7 and not h.value
    n = C.c_int32()
    assert lib.vp_rule_table(7, None, None, None, None, 64, C.byref(n)) == -1


@pytest.mark.parametrize("degree", [8, 12, 20, 25, 30, 40, 50])
def test_conical_rule_matches_oracle(degree):
    """The library generates the conical-product far rules on the host (long
    double), the oracle in 60-digit arithmetic: nodes and weights agree to one
    unit in the last place, w-hat and the degree exactly."""
    from oracle import gen_rules
    from paper_2205_04401_gb300 import vp
    x, y, w, what, deg = vp.far_rule(vp.VP_RULE_CONICAL(degree))
    r = gen_rules.conical_rule(degree)
    for a, k in ((x, "x"), (y, "y"), (w, "w")):
        b = np.array(r[k])
        assert len(a) == len(b)
        assert np.all(np.abs(a - b) <= np.spacing(np.abs(b))), k
    assert what == r["what"] and deg == degree


@pytest.mark.parametrize("degree", [12, 20, 25, 30, 40, 50])
def test_symmetric_rule_matches_oracle(tables, degree):
    """The library's S3-symmetric far rules (its own generator: invariants
    e2, e3 with rational moments) equal the oracle's (power sums p2, p3 with
    Gauss moments) bit for bit, w-hat included."""
    from paper_2205_04401_gb300 import vp
    x, y, w, what, deg = vp.far_rule(vp.VP_RULE_SYM(degree))
    r = tables[f"sym{degree}"]
    assert np.array_equal(x, r["x"]) and np.array_equal(y, r["y"]) and np.array_equal(w, r["w"])
    assert what == r["what"] and deg == degree


def test_far_rule_codes():
    from paper_2205_04401_gb300 import vp
    x, y, w, what, deg = vp.far_rule(vp.VP_RULE_19_D9)
    assert len(w) == 19 and deg == 9
    for bad in (17, vp.VP_RULE_CONICAL(7), vp.VP_RULE_CONICAL(51), vp.VP_RULE_SYM(13), vp.VP_RULE_SYM(8)):
        with pytest.raises(vp.VPError):
            vp.far_rule(bad)
