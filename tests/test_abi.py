"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/lsba.h (no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lsba.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lsba_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2208_09899_gb300 import build, lsba
    build.build()
    return lsba.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("lsba_create", "lsba_solve", "lsba_destroy", "lsba_get_stats", "lsba_status_string",
              "lsba_spmm", "lsba_gram", "lsba_combine"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2208_09899_gb300 import lsba
    so = lsba.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (lsba_\w+)", out))
    for n in _declared():
        assert n in exported, n
        assert hasattr(lib, n)
    assert set(lsba.EXPORTED) == set(_declared())


def test_status_strings_and_defaults(lib):
    import ctypes as C

    from paper_2208_09899_gb300 import lsba
    assert lsba.status_string(0) == "ok"
    assert "not converged" in lsba.status_string(1)
    o = lsba.Options()
    lib.lsba_default_options(C.byref(o))
    assert o.modification == 1 and o.max_restarts == 50 and o.adaptive_restart == 1
    assert o.inject_flag_cycle == -1


def test_invalid_arguments_without_gpu(lib):
    import ctypes as C
    assert lib.lsba_get_stats(None, None) == 3
    assert lib.lsba_destroy(None) == 3
    assert lib.lsba_create(None, 0, None, None) == 3
    # the autotuner and its table refuse a missing handle before any device work
    cnt = C.c_int(-1)
    assert lib.lsba_autotune(None, 1000, 8, 10, None, None, 0) == 3
    assert lib.lsba_autotune_table(None, None, 0, C.byref(cnt)) == 3 and cnt.value == -1


def test_binding_enums_match_header():
    """The binding's skeleton, modification and precision codes are the
    header's enumerators (the skeleton names are the paper's, lower case)."""
    from paper_2208_09899_gb300 import lsba
    src = open(os.path.join(ROOT, "include", "lsba.h")).read()
    body = re.search(r"typedef enum \{([^}]*)\} lsba_skeleton;", src).group(1)
    header = {m.group(1).lower(): int(m.group(2))
              for m in re.finditer(r"LSBA_(\w+)\s*=\s*(\d+)", body)}
    assert header == lsba.SKELETONS
    assert "bmgs" in header and "bcgsi_ls" in header


def _header_struct(name):
    """(type, field) pairs of `typedef struct { ... } name;` in lsba.h."""
    src = open(os.path.join(ROOT, "include", "lsba.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + ";", src).group(1)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        m = re.match(r"(.+?)\s*(\**)\s*(\w+)(\[\d+\])?$", decl)
        out.append((m.group(1).strip() + m.group(2), m.group(3), m.group(4)))
    return out


def test_binding_structs_match_header():
    """lsba_options, lsba_stats, lsba_history and lsba_tune_entry: the ctypes structures of the
    binding have the header's fields, in order, with the same sizes (a
    mismatch would shift every later option silently)."""
    import ctypes as C
    from paper_2208_09899_gb300 import lsba
    for cname, pystruct in (("lsba_options", lsba.Options), ("lsba_stats", lsba.Stats),
                            ("lsba_history", lsba.History), ("lsba_tune_entry", lsba.TuneEntry)):
        hdr = _header_struct(cname)
        py = pystruct._fields_
        assert [f for _, f, _ in hdr] == [f for f, _ in py], cname
        for (ctype, field, arr), (pf, pt) in zip(hdr, py):
            if ctype.endswith("*"):
                assert C.sizeof(pt) == C.sizeof(C.c_void_p), (cname, field)
            else:
                base = ctype.replace("const ", "")
                n = int(arr[1:-1]) if arr else 1
                size = {"int32_t": 4, "int64_t": 8, "double": 8, "float": 4}[base] * n
                assert C.sizeof(pt) == size, (cname, field)
