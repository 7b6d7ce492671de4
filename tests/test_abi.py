"""The C ABI library builds, loads and exports what include/hjm.h declares.

No compute call runs here (no GPU in this environment): only symbol lookup,
status strings and the host-side argument validation, which rejects bad
inputs before touching a device.
"""
import os
import re

import pytest

from paper_1108_1688_gb300 import _build
from paper_1108_1688_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    _build.build()
    from paper_1108_1688_gb300 import hjm
    return hjm


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hjm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hjm_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(H):
    names = declared_functions()
    assert len(names) >= 9
    for name in names:
        assert hasattr(H.lib, name), name
    assert set(names) == set(H.EXPORTED)


def test_status_strings(H):
    assert H.hjm_status_string(H.HJM_OK) == "ok"
    assert H.hjm_status_string(H.HJM_ERANGE) == "size out of supported range"
    assert H.hjm_status_string(99) == "unknown status"


@pytest.mark.parametrize("part,key,val,status", [
    ("grid", "n_r", 4, 1), ("grid", "n_r", 600, 7), ("grid", "n_v", 4000, 7),
    ("grid", "y_boundary_order", 0, 1), ("model", "rho", -1.5, 1), ("model", "gamma", 2.0, 1),
    ("inst", "T", -1.0, 1), ("curve", "kind", 7, 1), ("grid", "theta_adi", float("inf"), 1),
    ("grid", "scheme", 4, 1), ("grid", "scheme", -1, 1),
])
def test_batch_validation_rejects_bad_items(H, part, key, val, status):
    items = W.config2_draws(3, n_r=16, n_y=8, n_v=8, n_steps=4)
    items[1][part][key] = val
    with pytest.raises(H.HJMError) as ei:
        H.hjm_price_batch(items, H.HJM_FP32)
    assert ei.value.status == status
    assert "item 1" in str(ei.value)


@pytest.mark.parametrize("mutate", [
    lambda c: c.update(n_knots=0), lambda c: c.update(n_knots=33),
    lambda c: c["knot_t"].__setitem__(2, c["knot_t"][1]), lambda c: c["knot_P"].__setitem__(0, -0.1),
    lambda c: c["knot_t"].__setitem__(0, 0.0), lambda c: c["knot_P"].__setitem__(4, float("nan")),
])
def test_batch_validation_rejects_bad_knots(H, mutate):
    # the host-side checks of a discrete curve (no device is touched)
    items = W.config2_draws(2, n_r=16, n_y=8, n_v=8, n_steps=4)
    c = W.synthetic_knot_curve(3)
    mutate(c)
    items[1]["curve"] = c
    with pytest.raises(H.HJMError) as ei:
        H.hjm_price_batch(items, H.HJM_FP32)
    assert ei.value.status == H.HJM_EINVAL and "item 1" in str(ei.value)


def test_gamma_positive_needs_rmin_zero(H):
    it = W.paper_2007_set()
    it["grid"]["r_min"] = -0.01
    with pytest.raises(H.HJMError) as ei:
        H.hjm_grid_create(it["curve"], it["model"], it["grid"])
    assert ei.value.status == H.HJM_EINVAL


def test_empty_batch_is_a_no_op(H):
    assert len(H.hjm_price_batch([], H.HJM_FP32)) == 0


def test_struct_layout_matches_header(H, tmp_path):
    # Compile a probe against include/hjm.h with the host C compiler and
    # compare every struct's size and field offsets with the ctypes mirror.
    import ctypes as C
    import subprocess
    structs = {"hjm_curve": H.hjm_curve, "hjm_model_params": H.hjm_model_params,
               "hjm_grid_spec": H.hjm_grid_spec, "hjm_instrument": H.hjm_instrument,
               "hjm_price_info": H.hjm_price_info, "hjm_batch_item": H.hjm_batch_item}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hjm.h"', 'int main(void){']
    for cname, t in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in t._fields_:
            cf = "lambda" if fname == "lambda_" else fname
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, cf))
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    for line in filter(None, out):
        cname, fname, val = line.split()
        t = structs[cname]
        if fname == "size":
            assert C.sizeof(t) == int(val), cname
        else:
            assert getattr(t, fname).offset == int(val), (cname, fname)
