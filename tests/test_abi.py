"""The C ABI library loads and exports what include/tuckersinr.h declares;
host-side argument checks (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

from paper_2401_09792_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tuckersinr.h")


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    from paper_2401_09792_gb300 import tuckersinr as ts
    return ts.load(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ts_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ts_sinr_svd", "ts_sinr_mmse", "ts_workspace_bytes", "ts_status_string",
                     "ts_coefficients", "ts_project_precoder"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_the_header():
    from paper_2401_09792_gb300 import tuckersinr as ts
    for name in declared_functions():
        assert name in ts._SIG, f"binding lacks {name}"


def test_status_strings(lib):
    assert lib.ts_status_string(0) == b"ok"
    assert b"workspace" in lib.ts_status_string(4)
    assert lib.ts_abi_version() >= 1


def _dims(**kw):
    from paper_2401_09792_gb300 import tuckersinr as ts
    base = dict(J=2, M=4, N=32, P=8, m=4, n=8, p=4, K=64, L=2, delta_f_hz=15e3)
    base.update(kw)
    return ts.ts_dims(**base)


def test_workspace_sizes(lib):
    d = _dims()
    nch, P, K, n, L, p, m = 4, 8, 64, 8, 2, 4, 4
    svd = lib.ts_workspace_bytes(ctypes.byref(d), 0)
    mmse = lib.ts_workspace_bytes(ctypes.byref(d), 1)
    assert svd >= nch * P * 8 + 2 * K * n * L * 8 + 2 * K
    assert mmse >= nch * P * 8 + nch * p * m * L * 8
    assert svd % 256 == 0 and mmse % 256 == 0
    assert lib.ts_workspace_bytes(ctypes.byref(d), 99) == 0
    # several UEs per cell: two single-UE workspaces, whatever U
    assert lib.ts_workspace_bytes(ctypes.byref(d), 12) == 2 * svd
    assert lib.ts_workspace_bytes(ctypes.byref(d), 13) == 2 * lib.ts_workspace_bytes(ctypes.byref(d), 2)
    # the fit per model: the summed-Gram buffers grow with the number of factors
    # (shared 1, groupwise J, individual J^2); the reconstruction holds the two
    # intermediate products G x_1 A and (G x_1 A) x_2 B
    fit = [lib.ts_workspace_bytes(ctypes.byref(d), op) for op in (9, 6, 10)]
    assert 0 < fit[0] <= fit[1] <= fit[2]
    rec = lib.ts_workspace_bytes(ctypes.byref(d), 11)
    M, N = 4, 32
    assert rec >= nch * p * M * n * 8 + nch * p * M * N * 8
    # tensor-core modes: the svd workspace plus the rewritten core (per link:
    # TF32 2p K-elements of 4 bytes, BF16X2 6p of 2 bytes, per accumulator
    # column 2 MG n)
    tf32 = lib.ts_workspace_bytes(ctypes.byref(d), 7)
    bf16 = lib.ts_workspace_bytes(ctypes.byref(d), 8)
    assert tf32 >= svd + nch * (2 * m * n) * (2 * p) * 4
    assert bf16 >= svd + nch * (2 * m * n) * (6 * p) * 2


def test_tensor_core_operand_layout(lib):
    """The tensor-core workspace beyond the svd one, on the default system
    (J = 2, m = 4 -> 4-row lane groups, n = 8, p = 4, L = 2, K = 64): 128
    accumulator columns per block hold 128 / (2 * 4) = 16 columns of H~, so
    one block per link and one 128-subcarrier tile; an operand row holds the
    2p = 8 K-elements per segment (TF32: 4 bytes, one segment; TF32X3: hi and
    lo).  Core: J^2 links x 1 block x 128 rows; projections: J (J - 1)
    interfering links x 1 tile x 128 rows, and with TF32X3 also J serving
    links; precoder rows: J BSs x 1 tile x 1 block x 128 subcarriers x
    (16 columns x L = 32) complex, a whole number of 8-piece rows."""
    d = _dims()
    svd = lib.ts_workspace_bytes(ctypes.byref(d), 0)
    J, rows, vtile = 2, 128, 128 * 16 * 2 * 8
    for op, kbytes, serving in ((7, 8 * 4, 0), (14, 2 * 8 * 4, J)):
        core = J * J * rows * kbytes
        proj = (J * (J - 1) + serving) * rows * kbytes
        assert lib.ts_workspace_bytes(ctypes.byref(d), op) - svd == core + proj + J * vtile, op


def test_wide_cores_only_on_the_svd_path(lib):
    # p > 32 or P p > 8192: the SVD path streams the core (wide-core kernel);
    # the wideband-precoder path, the adjoints and the tensor-core modes stage
    # C_ik whole and refuse such sizes
    for kw in (dict(p=33, P=40), dict(p=20, P=512), dict(p=256, P=401, n=8)):
        d = _dims(**kw)
        assert lib.ts_workspace_bytes(ctypes.byref(d), 0) > 0, kw
        for op in (1, 4, 5, 7, 8):
            assert lib.ts_workspace_bytes(ctypes.byref(d), op) == 0, (kw, op)
    # the dense comparator keeps no projections: P up to 1024
    d = _dims(P=1024, p=4)
    assert lib.ts_workspace_bytes(ctypes.byref(d), 2) > 0
    assert lib.ts_workspace_bytes(ctypes.byref(d), 3) == 0


def test_tensor_core_modes_reject_unsupported_shapes(lib):
    from paper_2401_09792_gb300 import tuckersinr as ts
    d = _dims(M=16, m=16, L=16, N=32, n=16)
    assert lib.ts_workspace_bytes(ctypes.byref(d), 0) > 0
    assert lib.ts_workspace_bytes(ctypes.byref(d), 7) == 0
    coef = ts.ts_coef(0, 8, None, None)
    # L > 8 and unknown precisions are refused before any launch
    assert lib.ts_sinr_svd_prec(ctypes.byref(d), ctypes.byref(coef), 8, 8, 8, 1, 8, None, 256,
                                1 << 30, None) == 6
    d = _dims()
    assert lib.ts_sinr_svd_prec(ctypes.byref(d), ctypes.byref(coef), 8, 8, 8, 5, 8, None, 256,
                                1 << 30, None) == 6


@pytest.mark.parametrize("bad", [dict(m=5), dict(L=5), dict(L=0), dict(m=65, M=65),
                                 dict(n=33), dict(p=9), dict(p=257, P=300), dict(P=1025),
                                 dict(K=0), dict(J=0)])
def test_invalid_dims_rejected_before_launch(lib, bad):
    d = _dims(**bad)
    assert lib.ts_workspace_bytes(ctypes.byref(d), 0) == 0
    from paper_2401_09792_gb300 import tuckersinr as ts
    coef = ts.ts_coef(0, 8, None, None)
    st = lib.ts_sinr_svd(ctypes.byref(d), ctypes.byref(coef), 8, 8, 8, 8, None, 256, 1 << 30, None)
    assert st == 1


def test_null_and_alignment_checks(lib):
    from paper_2401_09792_gb300 import tuckersinr as ts
    d = _dims()
    coef = ts.ts_coef(0, None, None, None)
    assert lib.ts_sinr_svd(ctypes.byref(d), ctypes.byref(coef), 8, 8, 8, 8, None, 256, 1 << 30, None) == 2
    coef = ts.ts_coef(0, 8, None, None)
    assert lib.ts_sinr_svd(ctypes.byref(d), ctypes.byref(coef), 12, 8, 8, 8, None, 256, 1 << 30, None) == 3
    assert lib.ts_sinr_svd(ctypes.byref(d), ctypes.byref(coef), 8, 8, 8, 8, None, 256, 16, None) == 4
    assert lib.ts_sinr_svd(ctypes.byref(d), ctypes.byref(coef), 8, 8, 8, 8, None, 264, 1 << 30, None) == 3
    coef = ts.ts_coef(3, 8, None, None)
    assert lib.ts_sinr_svd(ctypes.byref(d), ctypes.byref(coef), 8, 8, 8, 8, None, 256, 1 << 30, None) == 6


def _instance(ts, **kw):
    d = _dims(**kw)
    coef = ts.ts_coef(1, None, 8, 8)
    return ts.ts_instance(d, 0, 0, coef, 8, 8, None, 8, 256, None)


def test_batch_workspace_and_checks_before_launch(lib, tmp_path):
    from paper_2401_09792_gb300 import tuckersinr as ts
    good = [_instance(ts), _instance(ts, K=100, J=3)]
    arr = (ts.ts_instance * 2)(*good)
    total = lib.ts_batch_workspace_bytes(arr, 2)
    each = [lib.ts_workspace_bytes(ctypes.byref(x.d), 0) for x in good]
    assert total == sum((b + 255) // 256 * 256 for b in each)      # two branches, one each
    # instances j and j + 4 share branch j's slot: its size is their maximum
    six = [_instance(ts, K=10 + 20 * j) for j in range(6)]
    arr6 = (ts.ts_instance * 6)(*six)
    b6 = [lib.ts_workspace_bytes(ctypes.byref(x.d), 0) for x in six]
    slots = [max(b6[j] for j in range(6) if j % 4 == b) for b in range(4)]
    assert lib.ts_batch_workspace_bytes(arr6, 6) == sum((b + 255) // 256 * 256 for b in slots)
    bad = (ts.ts_instance * 2)(good[0], _instance(ts, m=5))
    assert lib.ts_batch_workspace_bytes(bad, 2) == 0
    h = ctypes.c_void_p()
    # invalid sizes, an MMSE instance without precoder, a tensor-core MMSE
    # instance and a short workspace are refused before any CUDA call
    assert lib.ts_batch_plan_create(bad, 2, 256, 1 << 40, 0, ctypes.byref(h)) == 1
    mm = _instance(ts)
    mm.op = 1
    assert lib.ts_batch_plan_create((ts.ts_instance * 1)(mm), 1, 256, 1 << 40, 0, ctypes.byref(h)) == 2
    mm.Pt = 8
    mm.precision = 1
    assert lib.ts_batch_plan_create((ts.ts_instance * 1)(mm), 1, 256, 1 << 40, 0, ctypes.byref(h)) == 6
    assert lib.ts_batch_plan_create(arr, 2, 256, total - 1, 0, ctypes.byref(h)) == 4
    assert h.value is None


def test_autotune_table_roundtrip(lib, tmp_path):
    src = tmp_path / "in.txt"
    src.write_text("op0_prec0_J8_m8_n32_p16_P32_L8_K1024_coef1 2 1\nbroken line\n")
    assert lib.ts_autotune_load(str(src).encode()) == 0
    out = tmp_path / "out.txt"
    assert lib.ts_autotune_save(str(out).encode()) == 0
    assert "op0_prec0_J8_m8_n32_p16_P32_L8_K1024_coef1 2 1" in out.read_text()


def test_multiuser_checks_before_launch(lib):
    from paper_2401_09792_gb300 import tuckersinr as ts
    d = _dims()
    coef = ts.ts_coef(0, 8, None, None)
    single = lib.ts_workspace_bytes(ctypes.byref(d), ts.TS_OP_SINR_SVD)
    assert lib.ts_workspace_bytes(ctypes.byref(d), ts.TS_OP_SINR_SVD_MULTIUSER) == 2 * single
    f = lib.ts_sinr_svd_multiuser
    # no UE group; a missing core; one single-group workspace (two are needed)
    assert f(ctypes.byref(d), 0, ctypes.byref(coef), 8, 8, 8, 8, None, 256, 1 << 30, None) == 1
    assert f(ctypes.byref(d), 2, ctypes.byref(coef), None, 8, 8, 8, None, 256, 1 << 30, None) == 2
    assert f(ctypes.byref(d), 2, ctypes.byref(coef), 8, 8, 8, 8, None, 256, single, None) == 4
    g = lib.ts_dense_sinr_svd_multiuser
    assert g(ctypes.byref(d), 0, ctypes.byref(coef), 8, 8, 8, None, 256, 1 << 30, None) == 1
    assert g(None, 1, ctypes.byref(coef), 8, 8, 8, None, 256, 1 << 30, None) == 2


def test_fit_and_reconstruct_checks_before_launch(lib):
    from paper_2401_09792_gb300 import tuckersinr as ts
    # the fit takes ranks up to 256 (its eigensolver blocks); the
    # reconstruction any ranks up to the dimensions
    big = _dims(M=8, m=8, N=300, n=257, P=8, p=4)
    for op in (ts.TS_OP_TUCKER_FIT, ts.TS_OP_TUCKER_FIT_SHARED, ts.TS_OP_TUCKER_FIT_INDIVIDUAL):
        assert lib.ts_workspace_bytes(ctypes.byref(big), op) == 0
        assert lib.ts_workspace_bytes(ctypes.byref(_dims(n=8, N=300)), op) > 0
    assert lib.ts_workspace_bytes(ctypes.byref(big), ts.TS_OP_RECONSTRUCT) > 0
    d = _dims()
    fit = lib.ts_tucker_fit_model
    # oversized ranks, unknown model, negative sweep count, missing core,
    # misaligned factor, short workspace: all refused before any launch
    assert fit(ctypes.byref(big), 8, 1, 0, 0, 8, 8, 8, 8, 8, 256, 1 << 30, None) == 1
    assert fit(ctypes.byref(d), 8, 1, 0, 3, 8, 8, 8, 8, 8, 256, 1 << 30, None) == 6
    assert fit(ctypes.byref(d), 8, -1, 0, 0, 8, 8, 8, 8, 8, 256, 1 << 30, None) == 6
    assert fit(ctypes.byref(d), 8, 1, 0, 0, 8, 8, 8, None, 8, 256, 1 << 30, None) == 2
    assert fit(ctypes.byref(d), 8, 1, 0, 0, 12, 8, 8, 8, 8, 256, 1 << 30, None) == 3
    assert fit(ctypes.byref(d), 8, 1, 0, 0, 8, 8, 8, 8, 8, 256, 16, None) == 4
    rec = lib.ts_tucker_reconstruct
    assert rec(ctypes.byref(d), 7, 8, 8, 8, 8, 8, 256, 1 << 30, None) == 6
    assert rec(ctypes.byref(d), 0, 8, 8, 8, 8, None, 256, 1 << 30, None) == 2
    assert rec(ctypes.byref(d), 0, 8, 8, 8, 8, 8, 256, 16, None) == 4
