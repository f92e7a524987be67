"""CPU tests of the C ABI: the library loads, exports every declared symbol, its
ctypes mirror matches the header's layout, and the host-only reduction agrees
with the oracle's."""
import ctypes as C
import math
import os
import re
import subprocess

import pytest

import paper_2501_16909_b300 as ifr
from paper_2501_16909_b300 import _abi
from oracle import reduction as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(ifr_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2501_16909_b300 import build

    build.build()
    return _abi.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "ifr_sweep" in names and "ifr_sensitivity" in names and len(names) >= 13
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (ifr_\w+)$", out, flags=re.M))
    missing = names - exported
    assert not missing, missing
    for n in names:
        getattr(lib, n)


def test_struct_layouts_match_header(tmp_path, lib):
    checks = []
    for S in _abi.STRUCTS:
        checks.append('printf("%s %%zu\\n", sizeof(%s));' % (S.__name__, S.__name__))
        for f, _ in S._fields_:
            checks.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (S.__name__, f, S.__name__, f))
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "ifr.h"\nint main(void){%s return 0;}\n'
                   % "\n".join(checks))
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for S in _abi.STRUCTS:
        assert int(got[S.__name__]) == C.sizeof(S), S.__name__
        for f, _ in S._fields_:
            assert int(got["%s.%s" % (S.__name__, f)]) == getattr(S, f).offset, (S.__name__, f)


def test_strerror_and_version(lib):
    assert lib.ifr_abi_version() == 4
    assert lib.ifr_strerror(0) == b"ok"
    assert b"deadline" in lib.ifr_strerror(-3)


def _mk_cells(spec):
    cells = []
    for d in spec:
        c = _abi.ifr_cell_result()
        c.victim, c.stressor, c.level, c.repeat = d["victim"], d["stressor"], d["level"], d["repeat"]
        c.timing.t_start_ns, c.timing.t_end_ns, c.timing.repeats = d["t_start"], d["t_end"], d["k"]
        c.stress.status = d.get("stress_status", 0)
        c.stress.blocks_active = d.get("stress_blocks_active", 0)
        c.stress.t_start_last_ns = d.get("stress_t_start_last", 0)
        c.stress.t_end_first_ns = d.get("stress_t_end_first", 0)
        c.valid = 1 if R.cell_valid(d) else 0
        cells.append(c)
    return cells


def _random_spec(seed):
    import random

    rnd = random.Random(seed)
    spec = []
    for v in range(2):
        base = rnd.randint(1000, 5000)
        for rep in range(rnd.choice([2, 3, 4])):
            spec.append(dict(victim=v, stressor=-1, level=0, repeat=rep, k=3, t_start=100,
                             t_end=100 + 3 * int(base * rnd.uniform(0.95, 1.05))))
            for r in range(3):
                for l in range(4):
                    dur = int(base * (1 + 0.3 * l * r * rnd.uniform(0.8, 1.2)))
                    t = 10_000
                    ok = rnd.random() > 0.1
                    spec.append(dict(victim=v, stressor=r, level=l, repeat=rep, k=3, t_start=t, t_end=t + 3 * dur,
                                     stress_status=0, stress_blocks_active=4 if l else 0,
                                     stress_t_start_last=t - 1 if ok else t + 1, stress_t_end_first=t + 3 * dur + 1))
    return spec


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_host_sensitivity_matches_oracle(lib, seed):
    spec = _random_spec(seed)
    cells = _mk_cells(spec)
    inten = [[0.2, 0.5, 0.9], [0.3, 0.6, 1.0], [0.1, 0.4, 0.7]]
    for v in range(2):
        for it in (None, inten):
            got = ifr.ifr_sensitivity(cells, v, 3, 3, it)
            want = R.sensitivity(spec, v, 3, 3, it)
            assert got["t0"] == want["t0"]
            assert math.isclose(got["noise"], want["noise"], rel_tol=1e-12)
            for r in range(3):
                for l in range(4):
                    assert ifr.isclose_nan(got["slowdown"][r][l], want["slowdown"][r][l])
                assert ifr.isclose_nan(got["S"][r], want["S"][r])
                assert ifr.isclose_nan(got["auc"][r], want["auc"][r], rel=1e-9)
            assert got["monotone"] == want["monotone"]
            assert (got["n_valid"], got["n_invalid"]) == (want["n_valid"], want["n_invalid"])


def test_host_sensitivity_rejects_bad_args(lib):
    out = _abi.ifr_sensitivity_out()
    assert lib.ifr_sensitivity(None, 0, 0, 1, 0, None, C.byref(out)) == _abi.IFR_ERR_ARG
    assert lib.ifr_sensitivity(None, 0, 0, 99, 2, None, C.byref(out)) == _abi.IFR_ERR_ARG
    assert lib.ifr_sensitivity(None, 0, 0, 1, 2, None, None) == _abi.IFR_ERR_ARG
