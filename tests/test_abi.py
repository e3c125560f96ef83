"""The C ABI library loads on a CPU-only host and exports every symbol that
include/mrdem.h declares; host-only calls work without a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "mrdem.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mrdem_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    import paper_2105_12415_gb300 as m
    lib = m.load()
    names = _declared()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(m._lib.SIGNATURES)


def test_binding_signatures_match_the_header():
    """Every ctypes signature of the binding takes as many arguments as the
    header's prototype (a mismatch would pass garbage through the ABI)."""
    import paper_2105_12415_gb300 as m
    txt = open(os.path.join(ROOT, "include", "mrdem.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    protos = dict(re.findall(r"\b(mrdem_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", txt, flags=re.S))
    assert set(protos) == set(m._lib.SIGNATURES)
    scalar = {"int64_t": C.c_int64, "int32_t": C.c_int32, "int": C.c_int, "double": C.c_double}
    for name, params in protos.items():
        params = params.strip()
        plist = [] if params in ("", "void") else [x.strip() for x in params.split(",")]
        args = m._lib.SIGNATURES[name][1]
        assert len(args) == len(plist), (name, len(plist))
        for decl, ct in zip(plist, args):
            if "*" in decl or decl.startswith("mrdem_stream"):
                # pointers (and the stream handle) travel as pointers
                assert ct in (C.c_void_p, C.c_char_p) or issubclass(ct, C._Pointer) or \
                    hasattr(ct, "contents"), (name, decl)
            else:
                base = decl.split()[0]
                assert base in scalar, (name, decl)
                assert C.sizeof(ct) == C.sizeof(scalar[base]) and \
                    (ct is C.c_double) == (base == "double"), (name, decl, ct)


def test_status_strings_and_defaults():
    import paper_2105_12415_gb300 as m
    lib = m.load()
    for s in (0, -1, -2, -3, -4, -5):
        assert lib.mrdem_status_string(s)
    p = m.default_params()
    assert p.n_iter == 4 and p.fanout == 8 and p.leaf_max == 32 and abs(p.conv_c - 1.0) < 1e-7


def test_create_without_gpu_reports_cuda_error():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2105_12415_gb300 as m
    h = C.c_void_p()
    assert m.load().mrdem_create(C.byref(h), 0, None) == m._lib.MRDEM_ERR_CUDA


def test_null_arguments_are_rejected():
    import paper_2105_12415_gb300 as m
    lib = m.load()
    assert lib.mrdem_create(None, 0, None) == m._lib.MRDEM_ERR_INVALID
    assert lib.mrdem_detect(None, None, 0, None, None, None, 0, None, None, None) == -1
    assert lib.mrdem_check(None, None, None) == -1
    assert lib.mrdem_merge_contacts(None, 0, None, None, None, None, None) == -1
    assert lib.mrdem_hier_get_info(None, None) == -1
    assert lib.mrdem_broad_phase(None, 0, None, None, None, 0.01, None, None, 0, None, None) == -1
    assert lib.mrdem_move_poses(None, 0, None, None, 1e-3, None, None) == -1
    g = (C.c_double * 3)(0.0, 0.0, -9.81)
    assert lib.mrdem_picard_update(None, 0, None, None, None, None, C.cast(g, C.c_void_p), 1e-3,
                                   None, None, None) == -1
    assert lib.mrdem_contact_hessian(None, None, 0, None, None, None, None, None, 1000.0, None,
                                     None, None) == -1
    assert lib.mrdem_newton_residual(None, 0, None, None, None, None, None,
                                     C.cast(g, C.c_void_p), 1e-3, None, None, None) == -1
    assert lib.mrdem_newton_solve(None, 0, 0, None, None, None, None, 1e-3, None, None, 10, 1e-10,
                                  0, None, None) == -1
    assert lib.mrdem_vel_axpy(None, 0, 1.0, None, None, None, None) == -1
    assert lib.mrdem_destroy(None) == 0


def test_plain_c_caller(tmp_path):
    """The boundary is a C ABI: a C program that includes only
    include/mrdem.h and links libmrdem.so builds trees on the host, has bad
    input rejected with a status, and (without a GPU) gets MRDEM_ERR_CUDA from
    mrdem_create."""
    import subprocess

    import torch
    import paper_2105_12415_gb300 as m
    lib = m._lib.library_path()
    m.load()
    exe = tmp_path / "c_abi_example"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c_abi_example.c"), "-o", str(exe),
                           "-L", os.path.dirname(lib), "-lmrdem",
                           "-Wl,-rpath," + os.path.dirname(lib)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "trees: 2 particles" in r.stdout
    if not torch.cuda.is_available():
        assert "no GPU here" in r.stdout


def test_status_words_decode_like_the_check():
    """mrdem_status_decode on hand-made status words: overflow counts go to
    `required` in mrdem_check's order and give CAPACITY, a non-finite input
    gives NONFINITE first, an overflowing active-set list gives CAPACITY."""
    import numpy as np
    import paper_2105_12415_gb300 as m
    lib = m.load()
    assert m._lib.MRDEM_STATUS_WORDS == 8

    def decode(words):
        w = np.asarray(words, np.uint64)
        req = np.full(5, -1, np.int64)
        st = lib.mrdem_status_decode(C.c_void_p(w.ctypes.data), C.c_void_p(req.ctypes.data))
        return st, req.tolist()
    assert decode([0] * 8) == (0, [0, 0, 0, 0, 0])
    assert decode([0, 7, 0, 0, 123, 0, 0, 0]) == (m._lib.MRDEM_ERR_CAPACITY, [7, 0, 0, 123, 0])
    assert decode([1, 0, 0, 5, 0, 0, 0, 0])[0] == m._lib.MRDEM_ERR_NONFINITE
    assert decode([0, 0, 0, 0, 0, 0, 9, 0])[0] == m._lib.MRDEM_ERR_CAPACITY
    assert lib.mrdem_status_decode(None, None) == m._lib.MRDEM_ERR_INVALID
