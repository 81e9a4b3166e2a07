"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/sbs.h declares; configuration validation needs no device."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2403_11383_b300 import build as B
from paper_2403_11383_b300 import sbs as S
from paper_2403_11383_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "sbs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sbs_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return S.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (sbs_[a-z0-9_]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    # and the Python binding marshals every one of them
    assert set(names) == set(S.ABI), set(names) ^ set(S.ABI)
    for n in names:
        getattr(lib, n)


def test_struct_sizes_match_header(tmp_path):
    # gcc computes the sizes of the ABI structs from the header itself
    code = r'''
#include <stdio.h>
#include "sbs.h"
int main(void) { printf("%zu %zu %zu %zu %zu %zu\n", sizeof(sbs_config), sizeof(sbs_problem),
  sizeof(sbs_result), sizeof(sbs_gait), sizeof(sbs_model), sizeof(sbs_cost)); return 0; }
'''
    tmp = os.path.join(tmp_path, "abi_sizes")
    with open(tmp + ".c", "w") as f:
        f.write(code)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", tmp, tmp + ".c"], check=True)
    got = [int(v) for v in subprocess.run([tmp], capture_output=True, text=True, check=True).stdout.split()]
    want = [C.sizeof(S.Config), C.sizeof(S.Problem), C.sizeof(S.Result), C.sizeof(S.Gait), C.sizeof(S.Model),
            C.sizeof(S.Cost)]
    assert got == want


def test_status_strings(lib):
    for s in (0, 1, -1, -2, -3, -4, -5, -6):
        assert S.status_str(s) not in ("", "unknown status")


@pytest.mark.parametrize("field,value", [("K", 0), ("H", 0), ("H", 129), ("P", 5), ("P", 1), ("method", 7),
                                         ("iterations", 0), ("elite_count", 0), ("dt_us", 0), ("lam", 0.0),
                                         ("f_max", 0.5), ("tile", 48), ("tile", 512), ("q_init", 0)])
def test_invalid_config_rejected_without_device(lib, field, value):
    c = S.make_config(W.config("adaptive_elite_k8192_h25"))
    setattr(c, field, value)
    h = C.c_void_p()
    assert lib.sbs_create(C.byref(c), None, C.byref(h)) == S.ERR_INVALID_ARG
    assert not h.value


def test_invalid_model_rejected_without_device(lib):
    cfg = W.config("plain_mppi_k512_h12")
    c = S.make_config(cfg)
    c.model.mass = -1.0
    h = C.c_void_p()
    assert lib.sbs_create(C.byref(c), None, C.byref(h)) == S.ERR_INVALID_ARG
    c = S.make_config(cfg)
    c.cost.Q[3] = -1.0
    assert lib.sbs_create(C.byref(c), None, C.byref(h)) == S.ERR_INVALID_ARG
    # a phase step of a full cycle per time step is rejected
    cfg2 = dict(cfg, dt_us=300000, f_max=4.0)
    c = S.make_config(cfg2)
    assert lib.sbs_create(C.byref(c), None, C.byref(h)) == S.ERR_INVALID_ARG


@pytest.mark.parametrize("change", [
    dict(method="mppi"), dict(method="elite", elite_count=10), dict(adaptive=True), dict(compare_mppi=True),
    dict(freq_set_mhz=(1300, 2000, 1300)), dict(freq_set_mhz=(0, 2000)), dict(freq_set_mhz=(1300, 20000)),
    dict(freq_set_mhz=tuple(range(1000, 1900, 100))),  # nine values
    dict(dt_us=500_000, f_max=1.5),  # 2.4 Hz advances the phase by more than a cycle per step
])
def test_invalid_frequency_set_rejected_without_device(lib, change):
    cfg = W.config("naive_freqset_k10000_h12")
    cfg.update(change)
    c = S.make_config(cfg)
    if len(cfg["freq_set_mhz"]) > S.MAX_FREQ:
        c.n_freq = len(cfg["freq_set_mhz"])
    h = C.c_void_p()
    assert lib.sbs_create(C.byref(c), None, C.byref(h)) == S.ERR_INVALID_ARG
    assert not h.value


def test_null_arguments(lib):
    assert lib.sbs_create(None, None, None) == S.ERR_INVALID_ARG
    assert lib.sbs_solve(None, None, None, None) == S.ERR_INVALID_ARG
    assert lib.sbs_batch_solve(None, 0, None, None, None, None) == S.ERR_INVALID_ARG
    assert lib.sbs_dim(None) == S.ERR_INVALID_ARG
    lib.sbs_destroy(None)
    lib.sbs_batch_destroy(None)


def test_packed_batch_arguments():
    # Packed copies the handles and problems into the C arrays once; edits made in
    # place are what sbs_batch_solve reads
    class Fake:
        def __init__(self, v):
            self.handle = C.c_void_p(v)

    ctls = [Fake(0x1000 + 16 * i) for i in range(5)]
    probs = []
    for i in range(5):
        p = S.Problem()
        p.x0, p.xref, p.shift = 0x2000 + i, 0x3000 + i, i % 2
        p.gait = S.make_gait(W.gait("trot", 1000 * i))
        probs.append(p)
    pk = S.Packed(ctls, probs)
    assert pk.n == 5 and [h for h in pk.handles] == [c.handle.value for c in ctls]
    for i in range(5):
        assert pk.problems[i].x0 == probs[i].x0 and pk.problems[i].gait.phase0 == 1000 * i
    pk.problems[3].gait.phase0 = 77
    raw = C.string_at(C.addressof(pk.problems) + 3 * C.sizeof(S.Problem), C.sizeof(S.Problem))
    assert S.Problem.from_buffer_copy(raw).gait.phase0 == 77
    assert probs[3].gait.phase0 == 3000  # the caller's objects are not aliased
    with pytest.raises(ValueError):
        S.Packed(ctls, probs[:4])
    with pytest.raises(ValueError):
        S.Packed([], [])


def test_tile_tuner_checks_its_arguments():
    from paper_2403_11383_b300 import tuning
    with pytest.raises(ValueError):
        tuning.tile_for_batch([], [])
    with pytest.raises(ValueError):
        tuning.tile_for_batch([W.config("plain_mppi_k512_h12")] * 2, [None])
