"""Host-side checks of the C ABI that need no GPU: the library loads, exports every function
declared in include/dufwi.h, and its host logic (validation, CFL limit, workspace sizing,
geometry checks) behaves as documented."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib_module():
    from paper_2603_04070_gb300 import build_lib
    build_lib.build()
    from paper_2603_04070_gb300 import dufwi
    return dufwi


def _declared_functions():
    with open(os.path.join(ROOT, "include", "dufwi.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(dufwi_\w+)\s*\(", text, flags=re.M)))


def test_library_exports_every_declared_symbol():
    d = _lib_module()
    names = _declared_functions()
    assert len(names) >= 8, names
    lib = ctypes.CDLL(d.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def test_binding_constants_match_the_header():
    """Every DUFWI_OPT_*, DUFWI_ERR_*, DUFWI_SNAP_*, DUFWI_BOUNDARY_* and DUFWI_FORWARD_* value the
    header defines is the one the binding uses, and the library knows every option."""
    import re
    d = _lib_module()
    header = open(os.path.join(ROOT, "include", "dufwi.h")).read()
    defs = dict(re.findall(r"#define DUFWI_((?:OPT|ERR)_[A-Z0-9_]+)\s+(-?\d+)", header))
    assert len([k for k in defs if k.startswith("OPT_")]) >= 10
    for k, v in defs.items():
        assert getattr(d, k) == int(v), k
    for k in (k for k in defs if k.startswith("OPT_")):
        d.get_option(getattr(d, k))                       # known to the library
    named = {"SNAP": d.SNAPSHOT_DTYPES, "BOUNDARY": d.BOUNDARIES, "FORWARD": d.FORWARD_PRECISIONS}
    enums = re.findall(r"#define DUFWI_(SNAP|BOUNDARY|FORWARD)_([A-Z0-9]+)\s+(\d+)", header)
    assert len(enums) == 7
    for group, name, v in enums:
        assert named[group][name.lower()] == int(v), (group, name)


def test_status_strings_and_version():
    d = _lib_module()
    for code in range(9):
        assert d.status_string(code) and d.status_string(code) != "unknown status"
    assert d.status_string(1234) == "unknown status"
    assert d.version() > 0


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_cfl_limit_matches_oracle_stencil(order):
    """2/sqrt(2 rho), with rho the magnitude of the oracle's 1-D stencil at Nyquist."""
    d = _lib_module()
    c = oracle.fd_coeffs(order)
    nyq = c[0] + 2 * sum(c[k] * (-1) ** k for k in range(1, c.size))
    assert d.cfl_limit(order) == pytest.approx(2.0 / np.sqrt(2 * abs(nyq)), rel=1e-12)
    assert d.cfl_limit(3) < 0


def _problem(d, **kw):
    base = dict(nx=64, nz=48, dx=1e-4, dt=1e-8, nt=100, pml_cells=20, fd_order=8, c_max=1700.0)
    base.update(kw)
    return d.Problem(**base)


def _geom(d, n_elem=8, n_tx=2, n_rx=8):
    ix = np.arange(n_elem, dtype=np.int32) * 3 + 10
    return d.Geometry(ix, np.zeros(n_elem, np.int32), np.arange(n_tx) * 3,
                      np.tile(np.arange(n_rx), (n_tx, 1)))


def test_workspace_size_validation():
    d = _lib_module()
    g = _geom(d)
    n1 = d.workspace_size(_problem(d), g, 1)
    n2 = d.workspace_size(_problem(d), g, 2)
    assert n2 > n1 > 0
    sim = d.workspace_size(_problem(d), g, 1, gradient=False)
    assert 0 < sim < n1
    # padded grid 104 x 88 -> pitch 104; 2 shots; fields alone exceed 2 * 2 * 88 * 104 * 4 bytes
    assert sim >= 2 * 2 * 88 * 104 * 4
    # checkpointing bounds the history to one segment
    full = d.workspace_size(_problem(d, nt=2000), g, 1)
    ck = d.workspace_size(_problem(d, nt=2000, ckpt_interval=50), g, 1)
    ck16 = d.workspace_size(_problem(d, nt=2000, ckpt_interval=50, snapshot_dtype="bf16"), g, 1)
    assert ck16 < ck < full
    with pytest.raises(d.DufwiError) as e:
        d.workspace_size(_problem(d, fd_order=5), g, 1)
    assert e.value.status == d.ERR_INVALID_ARG
    with pytest.raises(d.DufwiError) as e:
        d.workspace_size(_problem(d, dt=1e-7), g, 1)          # CFL 1.7 > 0.555
    assert e.value.status == d.ERR_CFL
    with pytest.raises(d.DufwiError) as e:
        d.workspace_size(_problem(d, nt=0), g, 1)
    assert e.value.status == d.ERR_INVALID_ARG
    with pytest.raises(d.DufwiError):
        d.workspace_size(_problem(d), g, 0)


def test_geometry_errors_are_reported_before_any_device_work():
    """An element outside the grid or an out-of-range element index fails on the host.
    The pointers are never dereferenced because validation precedes every CUDA call."""
    d = _lib_module()
    pb = _problem(d)
    fake = ctypes.c_void_p(1 << 20)
    for bad in ("ix", "elem"):
        g = _geom(d)
        if bad == "ix":
            g.elem_ix[3] = pb.nx          # one past the last column
        else:
            g.tx_elem[1] = 99             # element index out of range
        arr, sh = g.c_structs()
        c = pb.c_struct()
        need = d.workspace_size(pb, _geom(d), 1, gradient=False)
        rc = d._lib.dufwi_simulate(ctypes.byref(c), fake, None, ctypes.byref(arr), fake, ctypes.byref(sh), 1,
                                   fake, ctypes.c_void_p(1 << 20), need, None)
        assert rc == d.ERR_GEOMETRY
    # too-small or misaligned workspace
    g = _geom(d)
    arr, sh = g.c_structs()
    c = pb.c_struct()
    need = d.workspace_size(pb, g, 1, gradient=False)
    assert d._lib.dufwi_simulate(ctypes.byref(c), fake, None, ctypes.byref(arr), fake, ctypes.byref(sh), 1,
                                 fake, ctypes.c_void_p(1 << 20), need - 1, None) == d.ERR_WORKSPACE
    assert d._lib.dufwi_simulate(ctypes.byref(c), fake, None, ctypes.byref(arr), fake, ctypes.byref(sh), 1,
                                 fake, ctypes.c_void_p((1 << 20) + 4), need, None) == d.ERR_WORKSPACE


def test_boundary_and_option_validation():
    """Absorbing-layer selection and launch options are checked on the host."""
    d = _lib_module()
    g = _geom(d)
    damp = d.workspace_size(_problem(d), g, 1)
    cpml = d.workspace_size(_problem(d, boundary="cpml", pml_alpha=6e6), g, 1)
    assert cpml > damp                                   # memory variables and coefficient tables
    # checkpointed CPML gradients add the memory-field snapshots and the adjoint's own sets
    ck = d.workspace_size(_problem(d, nt=2001, boundary="cpml", ckpt_interval=50), g, 1)
    ck0 = d.workspace_size(_problem(d, nt=2001, ckpt_interval=50), g, 1)
    field = 2 * (48 + 40) * ((64 + 40 + 7) // 8 * 8) * 4
    assert ck - ck0 >= (8 + 8 + 39 * 4) * field              # 40 segments, the last one kept
    # the Born call with the CPML adds the Born field's two memory sets and one scratch field
    j_c = d.jvp_workspace_size(_problem(d, boundary="cpml", pml_alpha=6e6), g, 1)
    j_d = d.jvp_workspace_size(_problem(d), g, 1)
    assert j_c >= j_d + (8 + 8 + 1) * field
    with pytest.raises(d.DufwiError) as e:
        d.workspace_size(_problem(d, boundary="cpml", pml_alpha=-1.0), g, 1)
    assert e.value.status == d.ERR_INVALID_ARG
    bad = _problem(d).c_struct()
    bad.boundary = 7
    sh = g.c_structs()[1]
    out = ctypes.c_size_t(0)
    assert d._lib.dufwi_workspace_size(ctypes.byref(bad), ctypes.byref(sh), 1, ctypes.byref(out)) == d.ERR_INVALID_ARG
    for opt, good, badv in ((d.OPT_PERSISTENT, 1, 2), (d.OPT_TEST_STALL, 0, 3), (d.OPT_TILE_Z, 64, 48),
                            (d.OPT_SHOT_GROUPS, 4, 5), (d.OPT_SHOT_GROUPS, 1, 0), (d.OPT_MIN_CTAS, 6, 7),
                            (d.OPT_MIN_CTAS, 4, 3), (d.OPT_CLUSTER, 1, 2)):
        before = d.get_option(opt)
        with pytest.raises(d.DufwiError):
            d.set_option(opt, badv)
        d.set_option(opt, good)
        assert d.get_option(opt) == good
        d.set_option(opt, before)


def test_second_order_workspace_sizing_and_validation():
    """The second-order call keeps two histories: every step with ckpt_interval 0, one segment
    of each plus four FP32 snapshots per segment otherwise; with the CPML also the memory
    variables of its four fields (two sets of four each) and, checkpointed, U's and dU's memory
    sets at every segment start."""
    d = _lib_module()
    g = _geom(d)
    pb_all = _problem(d, nt=200)
    pb_ck = _problem(d, nt=200, ckpt_interval=20)
    n_all = d.second_order_workspace_size(pb_all, g, 1)
    n_ck = d.second_order_workspace_size(pb_ck, g, 1)
    field = 4 * 2 * (48 + 40) * ((64 + 40 + 7) // 8 * 8)          # S x nzp x pitch floats
    assert n_all >= 2 * 199 * field                                  # Lap(U^n), Lap(dU^n) for every step
    assert 2 * 20 * field + 10 * 4 * field <= n_ck < n_all
    assert d.second_order_workspace_size(pb_all, g, 3) > n_all
    c_all = d.second_order_workspace_size(_problem(d, nt=200, boundary="cpml", pml_alpha=6e6), g, 1)
    c_ck = d.second_order_workspace_size(_problem(d, nt=200, ckpt_interval=20, boundary="cpml", pml_alpha=6e6), g, 1)
    assert c_all >= n_all + 4 * 8 * field
    assert c_ck >= n_ck + 4 * 8 * field + 10 * 8 * field
    with pytest.raises(d.DufwiError) as e:
        d.second_order_workspace_size(_problem(d, nt=0), g, 1)
    assert e.value.status == d.ERR_INVALID_ARG


def test_second_order_entry_points_reject_bad_arguments_before_device_work():
    """dufwi_second_order / dufwi_hvp: a missing output or input, or a workspace below the layout's
    size (with the damping layer or the CPML), is reported by the return value before anything
    touches the device (dummy host pointers suffice)."""
    d = _lib_module()
    g = _geom(d)
    arr, sh = g.c_structs()
    pb = _problem(d).c_struct()
    buf = (ctypes.c_float * 16)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    lib = d._lib
    # so (output) missing
    assert lib.dufwi_second_order(ctypes.byref(pb), p, None, ctypes.byref(arr), p, ctypes.byref(sh), 1, p, p,
                                  None, None, None, p, 1 << 30, None) == d.ERR_INVALID_ARG
    # dsos missing
    assert lib.dufwi_second_order(ctypes.byref(pb), p, None, ctypes.byref(arr), p, ctypes.byref(sh), 1, p, None,
                                  None, p, None, p, 1 << 30, None) == d.ERR_INVALID_ARG
    # cd_grad missing with receivers
    assert lib.dufwi_second_order(ctypes.byref(pb), p, None, ctypes.byref(arr), p, ctypes.byref(sh), 1, None, p,
                                  None, p, None, p, 1 << 30, None) == d.ERR_INVALID_ARG
    # hv missing; cd_obs missing
    assert lib.dufwi_hvp(ctypes.byref(pb), p, None, ctypes.byref(arr), p, ctypes.byref(sh), 1, p, p, None, None,
                         None, p, 1 << 30, None) == d.ERR_INVALID_ARG
    assert lib.dufwi_hvp(ctypes.byref(pb), p, None, ctypes.byref(arr), p, ctypes.byref(sh), 1, None, p, p, None,
                         None, p, 1 << 30, None) == d.ERR_INVALID_ARG
    # the CPML layout (memory variables of every field) is larger still
    cp = _problem(d, boundary="cpml").c_struct()
    assert lib.dufwi_hvp(ctypes.byref(cp), p, None, ctypes.byref(arr), p, ctypes.byref(sh), 1, p, p, p, None,
                         None, p, 64, None) == d.ERR_WORKSPACE
    # a workspace below the layout's size is rejected before the tables are copied
    assert lib.dufwi_hvp(ctypes.byref(pb), p, None, ctypes.byref(arr), p, ctypes.byref(sh), 1, p, p, p, None,
                         None, p, 64, None) == d.ERR_WORKSPACE


def test_workspace_allocation_failure_is_reported_as_a_library_error(monkeypatch):
    """The library allocates nothing; the binding allocates the workspace. A fault-injecting
    allocator that runs out of memory makes the binding raise DufwiError(ERR_WORKSPACE) with the
    size it needed; other allocator errors pass through unchanged."""
    import torch
    d = _lib_module()
    g = _geom(d)
    pb = _problem(d)
    need = d.workspace_size(pb, g, 1)
    real_empty = torch.empty

    def oom(*a, **k):
        if k.get("dtype") is torch.uint8:
            raise torch.cuda.OutOfMemoryError("CUDA out of memory. Tried to allocate 1.00 GiB")
        return real_empty(*a, **k)

    monkeypatch.setattr(d.torch, "empty", oom)
    with pytest.raises(d.DufwiError) as e:
        d._workspace(pb, g, 1, True, None, "cpu")
    assert e.value.status == d.ERR_WORKSPACE and str(need) in str(e.value)

    def broken(*a, **k):
        raise RuntimeError("device-side failure of another kind")

    monkeypatch.setattr(d.torch, "empty", broken)
    with pytest.raises(RuntimeError, match="another kind"):
        d._workspace(pb, g, 1, True, None, "cpu")


def _header_text():
    with open(os.path.join(ROOT, "include", "dufwi.h")) as f:
        return re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)


def test_binding_constants_match_the_header():
    """Status codes, snapshot types, boundaries, options and the no-alloc scratch size: the
    binding's values are the header's."""
    d = _lib_module()
    defs = {m.group(1): m.group(2).strip() for m in re.finditer(r"^#define\s+DUFWI_(\w+)\s+(.+)$", _header_text(),
                                                                 flags=re.M)}
    for name, val in defs.items():
        if name == "H":
            continue
        v = eval(val.replace("u", ""), {})                                   # e.g. (64u << 20)
        if name.startswith("SNAP_"):
            assert d.SNAPSHOT_DTYPES[name[5:].lower()] == v, name
        elif name.startswith("BOUNDARY_"):
            assert d.BOUNDARIES[name[9:].lower()] == v, name
        elif name.startswith("FORWARD_"):
            assert d.FORWARD_PRECISIONS[name[8:].lower()] == v, name
        else:
            assert getattr(d, name) == v, name


def test_binding_argument_counts_match_the_header_prototypes():
    """Every declared function the binding gives argtypes to takes as many arguments as its
    prototype has parameters (a mismatch would pass garbage through ctypes silently)."""
    d = _lib_module()
    text = _header_text()
    protos = {}
    for m in re.finditer(r"\b(dufwi_\w+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
        params = m.group(2).strip()
        protos[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    checked = 0
    for name, n in protos.items():
        fn = getattr(d._lib, name)
        if getattr(fn, "argtypes", None) is not None:
            assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)
            checked += 1
    assert checked >= 20


def test_problem_struct_layout_matches_the_header(tmp_path):
    """The ctypes mirror of dufwi_problem has the C struct's size and field offsets (a C program
    compiled against include/dufwi.h prints them), so no field is passed at the wrong place."""
    import subprocess
    d = _lib_module()
    fields = [f[0] for f in d._Problem._fields_]
    src = tmp_path / "layout.c"
    body = "".join('printf("%%s %%zu\\n", "%s", offsetof(dufwi_problem, %s));' % (f, f) for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "dufwi.h"\nint main(void){%s'
                   'printf("sizeof %%zu\\n", sizeof(dufwi_problem));return 0;}\n' % body)
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().split("\n") if line)
    assert int(out.pop("sizeof")) == ctypes.sizeof(d._Problem)
    for f in fields:
        assert int(out[f]) == getattr(d._Problem, f).offset, f


def test_compensated_forward_validation_and_sizing():
    """The compensated forward mode adds two low planes, kappa' / s_R as hi + lo and the low
    parts of the traces, and four-plane FP32 snapshots; it is refused on the host for the CPML,
    the Born and second-order calls, and unknown precision values."""
    d = _lib_module()
    g = _geom(d)
    field = 2 * (48 + 40) * ((64 + 40 + 7) // 8 * 8) * 4          # S x nzp x pitch floats, bytes
    for grad in (False, True):
        plain = d.workspace_size(_problem(d), g, 1, gradient=grad)
        comp = d.workspace_size(_problem(d, forward_precision="compensated"), g, 1, gradient=grad)
        assert comp >= plain + 2 * field + field                     # low planes + kq (two half-size maps)
    # FP32 snapshots: four planes per segment instead of two
    ck = dict(nt=2001, ckpt_interval=100)
    gap_fp32 = (d.workspace_size(_problem(d, forward_precision="compensated", **ck), g, 1)
                - d.workspace_size(_problem(d, **ck), g, 1))
    gap_fp16 = (d.workspace_size(_problem(d, forward_precision="compensated", snapshot_dtype="fp16", **ck), g, 1)
                - d.workspace_size(_problem(d, snapshot_dtype="fp16", **ck), g, 1))
    assert gap_fp32 - gap_fp16 >= 19 * 2 * field             # 20 segments, the last one kept
    for kw in (dict(boundary="cpml"),):
        with pytest.raises(d.DufwiError) as e:
            d.workspace_size(_problem(d, forward_precision="compensated", **kw), g, 1)
        assert e.value.status == d.ERR_UNSUPPORTED
    for fn in (d.jvp_workspace_size, d.second_order_workspace_size):
        with pytest.raises(d.DufwiError) as e:
            fn(_problem(d, forward_precision="compensated"), g, 1)
        assert e.value.status == d.ERR_UNSUPPORTED
    bad = _problem(d).c_struct()
    bad.forward_precision = 2
    sh = g.c_structs()[1]
    out = ctypes.c_size_t(0)
    assert d._lib.dufwi_workspace_size(ctypes.byref(bad), ctypes.byref(sh), 1, ctypes.byref(out)) == d.ERR_INVALID_ARG


def test_hybrid_history_workspace_sizing():
    """kept_segments = k keeps k segments of history (k K fields) and drops their snapshots; k at or
    above the segment count keeps every step and takes no snapshots; negative k is refused."""
    d = _lib_module()
    g = _geom(d)
    field = 2 * (48 + 40) * ((64 + 40 + 7) // 8 * 8) * 4
    K, nt = 50, 1001                                     # 20 segments
    base = d.workspace_size(_problem(d, nt=nt, ckpt_interval=K), g, 1)
    k1 = d.workspace_size(_problem(d, nt=nt, ckpt_interval=K, kept_segments=1), g, 1)
    assert base == k1                                        # the last segment is always kept
    k5 = d.workspace_size(_problem(d, nt=nt, ckpt_interval=K, kept_segments=5), g, 1)
    kall = d.workspace_size(_problem(d, nt=nt, ckpt_interval=K, kept_segments=20), g, 1)
    kmore = d.workspace_size(_problem(d, nt=nt, ckpt_interval=K, kept_segments=500), g, 1)
    store_all = d.workspace_size(_problem(d, nt=nt, ckpt_interval=0), g, 1)
    plain = d.workspace_size(_problem(d, nt=nt, ckpt_interval=K, snapshot_dtype="fp32"), g, 1)
    assert plain == base
    assert abs(k5 - k1 - 4 * K * field + 4 * 2 * field) <= 4096
    assert kall == kmore
    assert abs(kall - store_all) <= K * field + 4096          # 20 K slots against nt - 1 = 1000 steps
    assert d.workspace_size(_problem(d, nt=nt, ckpt_interval=0, kept_segments=3), g, 1) == store_all
    with pytest.raises(d.DufwiError) as e:
        d.workspace_size(_problem(d, nt=nt, ckpt_interval=K, kept_segments=-1), g, 1)
    assert e.value.status == d.ERR_INVALID_ARG


def test_kept_segments_for_budget_is_the_largest_fit():
    from paper_2603_04070_gb300 import autotune
    d = _lib_module()
    g = _geom(d)
    pb = _problem(d, nt=1001, ckpt_interval=50)
    sizes = [d.workspace_size(_problem(d, nt=1001, ckpt_interval=50, kept_segments=k), g, 1) for k in range(21)]
    assert all(a <= b for a, b in zip(sizes[1:], sizes[2:]))
    for k in (2, 7, 20):
        assert autotune.kept_segments_for_budget(pb, g, 1, sizes[k]) == k
        assert autotune.kept_segments_for_budget(pb, g, 1, sizes[k] - 1) == k - 1
    assert sizes[0] == sizes[1]
    assert autotune.kept_segments_for_budget(pb, g, 1, sizes[1] - 1) == 0
    assert autotune.kept_segments_for_budget(_problem(d, nt=1001, ckpt_interval=0), g, 1, 1 << 40) == 0


def test_autotune_candidates_are_valid_option_sets():
    """Every launch form the tuner times is a set of valid option values (host-side round trip),
    and applying a set changes only the eight launch options."""
    from paper_2603_04070_gb300 import autotune
    d = _lib_module()
    opts = {"tile_z": d.OPT_TILE_Z, "two_step": d.OPT_TWO_STEP, "persistent": d.OPT_PERSISTENT,
            "multi_tile": d.OPT_MULTI_TILE, "early": d.OPT_EARLY_LOADS, "groups": d.OPT_SHOT_GROUPS,
            "min_ctas": d.OPT_MIN_CTAS, "cluster": d.OPT_CLUSTER}
    assert set(autotune.KNOBS) == set(opts)
    before = {k: d.get_option(o) for k, o in opts.items()}
    reuse = d.get_option(d.OPT_REUSE_TABLES)
    try:
        for cand in autotune.CANDIDATES:
            autotune.apply(cand)
            assert {k: d.get_option(o) for k, o in opts.items()} == cand
            assert d.get_option(d.OPT_REUSE_TABLES) == reuse
        assert len({tuple(sorted(c.items())) for c in autotune.CANDIDATES}) == len(autotune.CANDIDATES)
    finally:
        autotune.apply(before)
    assert {k: d.get_option(o) for k, o in opts.items()} == before


def test_autotune_skips_candidates_that_do_not_apply():
    """The cluster form applies only to grids whose fields fit a cluster's shared memory (and not
    to maps of different sizes), the register-cap variants only to the 8th-order 64 x 32 form; the
    tuner does not time such candidates."""
    from paper_2603_04070_gb300 import autotune
    d = _lib_module()
    small = d.Problem(nx=128, nz=128, dx=1e-4, dt=1e-8, nt=10)
    ring = d.Problem(nx=188, nz=188, dx=1e-4, dt=1e-8, nt=10)
    big = d.Problem(nx=512, nz=512, dx=1e-4, dt=1e-8, nt=10)
    order4 = d.Problem(nx=128, nz=128, dx=1e-4, dt=1e-8, nt=10, fd_order=4)
    assert autotune.cluster_fits(small) and autotune.cluster_fits(ring) and not autotune.cluster_fits(big)
    cl = {**autotune._BASE, "cluster": 1}
    cap = {**autotune._BASE, "min_ctas": 4}
    assert autotune.applicable(cl, small) and not autotune.applicable(cl, big)
    assert not autotune.applicable(cl, small, sizes=[(128, 128)])
    assert autotune.applicable(cap, small) and not autotune.applicable(cap, order4)
    assert not autotune.applicable({**cap, "tile_z": 64}, small)
    assert all(autotune.applicable(c, small) for c in autotune.CANDIDATES)
