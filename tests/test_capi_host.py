"""Host-side checks of the C-ABI library (no GPU compute).

The library must load, export every function include/irk.h declares, reject
invalid configurations before touching a device, and compute the same
tableau and real Schur form as the oracle (up to the non-unique parts of a
Schur basis).
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_2101_01776_gb300 import build
    build.build()
    from paper_2101_01776_gb300 import binding
    return binding


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if not f.endswith(".h"):
            continue
        text = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, f)).read(), flags=re.S)
        names |= set(re.findall(r"\b(irk_[a-z_]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol(B):
    names = declared_functions()
    assert len(names) >= 12
    lib = ctypes.CDLL(B._LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(B.EXPORTED)


FAMILIES = [("gauss", 0, s) for s in (1, 2, 3, 4, 5)] + [("radau", 1, s) for s in (1, 2, 3, 4, 5)] \
    + [("lobatto", 2, s) for s in (2, 3, 4, 5)]


@pytest.mark.parametrize("family,fid,s", FAMILIES)
def test_host_tableau_matches_oracle(B, family, fid, s):
    from oracle import tableau as tab
    t = B.irk_tableau(s, fid)
    A, b, c = tab.tableau(family, s)
    np.testing.assert_allclose(t["A"], A, atol=1e-15)
    np.testing.assert_allclose(t["b"], b, atol=1e-15)
    np.testing.assert_allclose(t["c"], c, atol=1e-15)
    Ainv = np.linalg.inv(A)
    Q, R = t["Q0"], t["R0"]
    np.testing.assert_allclose(Q @ Q.T, np.eye(s), atol=1e-14)
    np.testing.assert_allclose(Q @ R @ Q.T, Ainv, atol=1e-12)
    # eta, beta^2 and gamma* per block agree with the oracle's Schur form
    Qo, Ro, blocks_o = tab.real_schur(Ainv)
    ours, k = [], 0
    for m in t["block_sizes"]:
        if m == 1:
            ours.append((round(R[k, k], 9), 0.0))
        else:
            assert abs(R[k, k] - R[k + 1, k + 1]) < 1e-13
            assert np.all(np.abs(R[k + 2:, k:k + 2]) == 0)
            ours.append((round(R[k, k], 9), round(-R[k, k + 1] * R[k + 1, k], 8)))
        k += m
    theirs = []
    for bc in tab.block_constants(Ro, blocks_o):
        theirs.append((round(bc["eta"], 9), round(bc["beta"] ** 2, 8)))
    assert sorted(ours) == sorted(theirs)


@pytest.mark.parametrize("family,fid,s", FAMILIES)
def test_host_eigen_basis_matches_oracle(B, family, fid, s):
    """Eigenvector basis: T R T^{-1} = A0^{-1}, Tinv = T^{-1}, R block diagonal
    with [[eta, beta], [-beta, eta]] blocks equal to the oracle's eigenvalues."""
    from oracle import tableau as tab
    A, _, _ = tab.tableau(family, s)
    Ainv = np.linalg.inv(A)
    e = B.irk_transform(s, fid, B.IRK_BASIS_EIGEN)
    T, Ti, R = e["T"], e["Tinv"], e["R"]
    np.testing.assert_allclose(T @ Ti, np.eye(s), atol=1e-13)
    np.testing.assert_allclose(T @ R @ Ti, Ainv, atol=1e-11)
    mask = np.zeros((s, s), bool)
    k = 0
    ours = []
    for m in e["block_sizes"]:
        mask[k:k + m, k:k + m] = True
        if m == 2:
            assert R[k, k] == R[k + 1, k + 1] and R[k, k + 1] == -R[k + 1, k] > 0
        ours.append((round(R[k, k], 9), round(R[k, k + 1], 9) if m == 2 else 0.0))
        k += m
    assert np.all(R[~mask] == 0)
    To, Ro, blocks = tab.real_eigen_basis(Ainv)
    theirs = [(round(Ro[k, k], 9), round(Ro[k, k + 1], 9) if m == 2 else 0.0) for (k, m) in blocks]
    assert ours == theirs  # same eigenvalue order: increasing real part
    # the Schur transform from the same entry point is orthogonal
    q = B.irk_transform(s, fid, B.IRK_BASIS_SCHUR)
    np.testing.assert_allclose(q["Tinv"], q["T"].T, atol=0)
    np.testing.assert_array_equal(q["T"], B.irk_tableau(s, fid)["Q0"])


def test_transform_rejects_bad_arguments(B):
    # (s, family, basis): bad basis, unknown family, s out of range, Lobatto s=1,
    # SDIRK without its 4-stage method, SDIRK in an eigenvector basis
    for args in [(2, 0, 2), (2, 4, 0), (0, 0, 0), (6, 0, 0), (1, 2, 0), (4, 3, 0), (2, 3, 1)]:
        with pytest.raises(B.IrkError):
            B.irk_transform(*args)


def test_gauss2_schur_basis_is_identity(B):
    """Eq. Gauss4Radau3_example: A0^{-1} of 2-stage Gauss is already in
    standardized form, so the block is exactly Newton (P-hat block diagonal)."""
    t = B.irk_tableau(2)
    np.testing.assert_array_equal(t["Q0"], np.eye(2))


def test_device_bytes_is_host_only_and_grows_with_the_problem(B):
    small = B.irk_config_default(op="burgers2d", n=64, stages=2)
    big = B.irk_config_default(op="burgers2d", n=256, stages=4)
    a, b = B.irk_config_device_bytes(small), B.irk_config_device_bytes(big)
    assert 0 < a < b
    assert B.irk_config_device_bytes(B.irk_config_default(stages=9)) == 0


def test_invalid_configs_rejected_before_device(B):
    u0 = np.zeros(256)
    bad = [dict(stages=0), dict(stages=6), dict(n=100), dict(nu=0.0), dict(nu=-1.0),
           dict(op="vsf", mass=0), dict(op="burgers1d", mass=1), dict(family=4),
           dict(family=3, stages=4), dict(family=3, stages=2, basis=1), dict(dirk_sequential=2),
           dict(dae_solver=2), dict(dae_solver=1), dict(dae_solver=-1),
           dict(initial_guess=3), dict(initial_guess=-1), dict(mg_tile_rows=7), dict(mg_tile_rows=-8),
           dict(family=-1), dict(family=2, stages=1), dict(basis=2), dict(basis=-1),
           dict(krylov_restart=0), dict(krylov_restart=65), dict(nonlinear_variant=5),
           dict(nonlinear_variant=-1), dict(mg_precision=3), dict(forcing=1, op="burgers2d"),
           dict(mg_shifted_sweeps=-1), dict(mg_shifted_sweeps=9), dict(mg_coarse_reduction=1.0),
           dict(mg_coarse_reduction=-0.1), dict(mg_coarse_smoother=3), dict(mg_coarse_smoother=-1),
           dict(mg_fuse_transfer=3), dict(mg_fuse_transfer=-1)]
    for kw in bad:
        cfg = B.irk_config_default(**kw)
        with pytest.raises(B.IrkError) as ei:
            B.irk_create(cfg, u0)
        assert ei.value.status == B.IRK_ERR_INVALID, kw


def test_no_device_reported_cleanly(B):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cfg = B.irk_config_default()
    with pytest.raises(B.IrkError) as ei:
        B.irk_create(cfg, np.zeros(256))
    assert ei.value.status == B.IRK_ERR_NO_DEVICE


@pytest.mark.parametrize("s", [1, 2, 3, 5])
def test_sdirk_tableau_and_exact_schur_form(B, s):
    """The library's SDIRK tableau (derived from the order conditions) equals
    the oracle's closed forms; its transform is the reversal permutation with
    R0 = J A0^{-1} J upper triangular, every block 1x1 with eta = 1/gamma."""
    from oracle import tableau as tab
    t = B.irk_tableau(s, B.IRK_SDIRK)
    A, b, c = tab.sdirk(s)
    # the oracle's 3-stage gamma is a double-precision polynomial root (a few
    # ulps); the library bisects the order-3 condition in long double
    np.testing.assert_allclose(t["A"], A, rtol=0, atol=1e-14)
    np.testing.assert_allclose(t["b"], b, rtol=0, atol=1e-14)
    np.testing.assert_allclose(t["c"], c, rtol=0, atol=1e-14)
    J = np.eye(s)[::-1]
    np.testing.assert_array_equal(t["Q0"], J)
    np.testing.assert_allclose(t["R0"], J @ np.linalg.inv(A) @ J, rtol=1e-14, atol=1e-13)
    assert list(t["block_sizes"]) == [1] * s
    q = B.irk_transform(s, B.IRK_SDIRK, B.IRK_BASIS_SCHUR)
    np.testing.assert_array_equal(q["Tinv"], J)


def test_sdirk_stage_by_stage_arena_holds_the_stage_solver(B):
    """A stage-by-stage SDIRK handle carves a single-stage solver out of its
    own arena; the coupled form needs no such second solver."""
    seq = B.irk_config_default(op="burgers2d", n=64, family="sdirk", stages=3)
    coupled = B.irk_config_default(op="burgers2d", n=64, family="sdirk", stages=3, dirk_sequential=0)
    one = B.irk_config_default(op="burgers2d", n=64, family="sdirk", stages=1)
    a, b, c = (B.irk_config_device_bytes(x) for x in (seq, coupled, one))
    assert 0 < c < b < a
    assert a >= b + c - 4096


def test_binding_refuses_short_buffers(B):
    """The library copies ncomp * n^dim values through the state pointer; the
    binding refuses a smaller buffer before calling it (a valid config only:
    invalid configs still reach the library's own checks)."""
    for kw, short in ((dict(op="burgers2d", n=64), np.zeros((2, 64, 63))),
                      (dict(op="vsf", n=32), np.zeros((1, 32, 32))),
                      (dict(op="burgers1d", n=256), np.zeros(255))):
        cfg = B.irk_config_default(**kw)
        with pytest.raises(ValueError, match="float64 values"):
            B.irk_create(cfg, short)
    # a right-sized state passes the binding (and fails on the missing device here)
    import torch
    if not torch.cuda.is_available():
        cfg = B.irk_config_default(op="burgers2d", n=64)
        with pytest.raises(B.IrkError):
            B.irk_create(cfg, np.zeros((2, 64, 64)))


def _c_struct_fields(header, typedef_name):
    """(name, C type) of each member of `typedef struct { ... } typedef_name;`
    in the header, in declaration order (comments removed; `a, b;` split)."""
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", header)).read(), flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + typedef_name + r"\s*;", text)
    assert m, typedef_name
    out = []
    for decl in m.group(1).split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        mm = re.match(r"((?:unsigned |long |const )*(?:long|int|double|char|size_t|float))\s+(.*)", decl)
        assert mm, decl
        ctype = mm.group(1)
        for name in mm.group(2).split(","):
            name = name.strip()
            arr = re.match(r"(\w+)\[(\d+)\]", name)
            out.append((arr.group(1), f"{ctype}[{arr.group(2)}]") if arr else (name, ctype))
    return out


@pytest.mark.parametrize("header,typedef,cls", [("irk.h", "irk_config", "IrkConfig"),
                                                ("irk.h", "irk_stats", "IrkStats"),
                                                ("irk.h", "irk_kernel_stat", "IrkKernelStat"),
                                                ("irk_serve.h", "irk_server_stats", "IrkServerStats")])
def test_binding_structs_mirror_the_headers(B, header, typedef, cls):
    """Every ctypes structure of the binding lists the header's members in the
    same order with the same C types, so the library and the binding agree on
    the layout (a mismatch would shift every later field)."""
    import ctypes
    want = _c_struct_fields(header, typedef)
    ctypes_of = {"int": ctypes.c_int, "double": ctypes.c_double, "long long": ctypes.c_longlong,
                 "size_t": ctypes.c_size_t, "float": ctypes.c_float}
    got = getattr(B, cls)._fields_
    assert [n for n, _ in got] == [n for n, _ in want], typedef
    for (name, ct), (_, t) in zip(want, got):
        if ct.startswith("char["):
            assert t._type_ is ctypes.c_char and t._length_ == int(ct[5:-1]), name
        else:
            assert t is ctypes_of[ct], (name, ct, t)


def test_config_defaults_are_the_documented_ones(B):
    """irk_config_default against the defaults the header documents for the
    solver's switches."""
    c = B.irk_config_default()
    assert (c.initial_guess, c.nonlinear_variant, c.dirk_sequential, c.dae_solver) == (2, 2, 1, 0)
    assert (c.mg_tile_rows, c.mg_fuse_transfer, c.mg_levels) == (0, 0, 0)
    assert c.use_graphs == 1 and c.newton_rtol == 1e-10


def test_batch_instance_bytes_accepts_only_the_batched_configurations(B):
    """irk_batch_instance_bytes (host-only) sizes an instance's arena for the
    batched 2D Burgers path and returns 0 for what it does not serve."""
    ok = B.irk_config_default(op="burgers2d", n=64, stages=3, nu=1e-2)
    small = B.IrkBatch.instance_bytes(ok)
    assert small > 0
    bigger = B.IrkBatch.instance_bytes(B.irk_config_default(op="burgers2d", n=128, stages=3, nu=1e-2))
    assert bigger > 3 * small
    more_stages = B.IrkBatch.instance_bytes(B.irk_config_default(op="burgers2d", n=64, stages=4, nu=1e-2))
    assert more_stages > small
    for kw in (dict(op="burgers1d", n=64), dict(op="vsf", n=64), dict(op="burgers2d", n=16),
               dict(op="burgers2d", n=64, mg_precision=1), dict(op="burgers2d", n=64, nonlinear_variant=3),
               dict(op="burgers2d", n=64, family="lobatto", stages=3),
               dict(op="burgers2d", n=64, krylov_restart=40), dict(op="burgers2d", n=96)):
        assert B.IrkBatch.instance_bytes(B.irk_config_default(**kw)) == 0, kw


def test_batch_create_without_a_device(B):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(B.IrkError) as ei:
        B.IrkBatch(4)
    assert ei.value.status == B.IRK_ERR_NO_DEVICE
