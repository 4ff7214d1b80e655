"""Host-side checks of the C ABI (no GPU needed).

The library must load and export every function that include/lbm_gb300.h
declares; the binding's structure layouts and constants must match the
header.  Nothing here launches a kernel.
"""
import ctypes as ct
import os
import re

import pytest

from paper_1702_04910_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm_gb300.h")


def header_text():
    with open(HEADER) as fh:
        return fh.read()


def declared_functions():
    src = re.sub(r"/\*.*?\*/", "", header_text(), flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    try:
        build.build()
    except RuntimeError as e:  # toolkit missing: the build check itself fails elsewhere
        pytest.skip(str(e))
    return ct.CDLL(build.LIB_PATH)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbm_create", "lbm_set_particles", "lbm_step", "lbm_get_forces",
                     "lbm_get_fields", "lbm_destroy"):
        assert required in names
    assert set(names) == set(binding.EXPORTED)


def test_library_exports_every_declared_function(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared but not exported"


def test_abi_version_without_gpu(lib):
    lib.lbm_abi_version.restype = ct.c_int
    assert lib.lbm_abi_version() == 1


def test_null_arguments_are_rejected_without_gpu(lib):
    """Argument validation happens before any CUDA call."""
    lib.lbm_create.restype = ct.c_int
    lib.lbm_create.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_void_p]
    assert lib.lbm_create(None, None, None) == binding.LBM_ERR_ARG
    cfg = binding.make_config((8, 8, 8), tau=0.4)  # tau <= 1/2 is invalid
    h = ct.c_void_p()
    assert lib.lbm_create(ct.byref(cfg), None, ct.byref(h)) == binding.LBM_ERR_ARG
    # MEM MR rebuilds its correction from post-collision values: refused where
    # Lambda_- = 1/2 (TRT: Lambda / (tau - 1/2) with Lambda = 3/16; BGK: tau - 1/2)
    for tau, coll in ((0.875, "TRT"), (0.88, "TRT"), (1.0, "BGK")):
        cfg = binding.make_config((8, 8, 8), coupling="MEM_MR", tau=tau, collision=coll)
        assert lib.lbm_create(ct.byref(cfg), None, ct.byref(h)) == binding.LBM_ERR_UNSUPPORTED
    cfg = binding.make_config((0, 8, 8))
    assert lib.lbm_create(ct.byref(cfg), None, ct.byref(h)) == binding.LBM_ERR_ARG
    lib.lbm_step.restype = ct.c_int
    lib.lbm_step.argtypes = [ct.c_void_p, ct.c_int]
    assert lib.lbm_step(None, 1) == binding.LBM_ERR_ARG
    # the re-mapping charge and the batch's bulk timing check their handle first
    for name in ("lbm_set_remap_charge", "lbm_batch_set_remap_charge", "lbm_batch_profile_enable"):
        fn = getattr(lib, name)
        fn.restype = ct.c_int
        fn.argtypes = [ct.c_void_p, ct.c_int]
        assert fn(None, 1) == binding.LBM_ERR_ARG, name
    lib.lbm_batch_profile_read.restype = ct.c_int
    lib.lbm_batch_profile_read.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_void_p]
    ms, n = ct.c_double(), ct.c_longlong()
    assert lib.lbm_batch_profile_read(None, ct.byref(ms), ct.byref(n)) == binding.LBM_ERR_ARG


def test_struct_layouts_match_header():
    """Field order and sizes of the two public structs (x86-64 / aarch64 LP64)."""
    assert ct.sizeof(binding.LbmParticle) == 11 * 8 + 8
    assert binding.LbmConfig.tau.offset == 24
    assert binding.LbmConfig.storage.offset == 108 and binding.LbmConfig.inflow.offset == 112
    assert binding.LbmConfig.rho_out.offset == 136 and ct.sizeof(binding.LbmConfig) == 144
    text = header_text()
    cfg_block = text[text.index("typedef struct {"):text.index("} lbm_config;")]
    fields = re.findall(r"\b(?:int|double)\s+([a-z_0-9\[\], ]+);", cfg_block)
    flat = []
    for f in fields:
        for name in f.split(","):
            flat.append(re.sub(r"\[.*\]", "", name).strip())
    assert flat == [n for n, _ in binding.LbmConfig._fields_]


def test_enum_values_match_header():
    text = header_text()
    for name, val in binding.COUPLING.items():
        assert re.search(rf"LBM_{name}\s*=\s*{val}\b", text), name
    for st, name in binding.STATUS_NAMES.items():
        assert re.search(rf"{name}\s*=\s*{st}\b", text), name
    for name, bit in binding.STATUS_BITS.items():
        assert re.search(rf"{name}\s*=\s*{bit}\b", text), name
    for name in ("PDF", "PDF_PRE", "RHO", "U", "EPS", "FLAG", "PDF_F64", "REMAP_CHARGE"):
        val = getattr(binding, f"FIELD_{name}")
        assert re.search(rf"LBM_FIELD_{name}\s*=\s*{val}\b", text), name


def test_binding_wrapper_surface():
    """The Python wrapper keeps the methods the tests and the benchmark use."""
    for name in ("set_particles", "get_particles", "init_equilibrium", "step", "forces",
                 "set_pdf_pre", "pdf", "pdf_f64", "set_pdf", "macro", "eps", "flags",
                 "synchronize", "close", "set_remap_charge", "remap_charge",
                 "set_remap_charge_state"):
        assert callable(getattr(binding.Simulation, name)), name
    for name in binding.EXPORTED:
        if name not in ("lbm_last_error", "lbm_abi_version", "lbm_batch_last_error",
                        "lbm_mlp_last_error"):
            assert callable(getattr(binding, name)), name
    for name in ("step", "autotune", "set_tuning", "particles", "forces", "pdf", "synchronize",
                 "close", "set_remap_charge", "profile", "profile_read"):
        assert callable(getattr(binding.Batch, name)), name


def test_batch_rejects_invalid_cases_without_gpu():
    """lbm_batch_create validates every case before any CUDA call and leaves
    the reason readable through lbm_batch_last_error(NULL)."""
    from paper_1702_04910_gb300 import workloads as W
    lib = binding.load()
    cases = W.ensemble(3, seed=1, d_range=(5, 6))

    def create(cfgs, parts):
        carr = (binding.LbmConfig * len(cfgs))(*cfgs)
        b = ct.c_void_p()
        st = lib.lbm_batch_create(len(cfgs), carr, binding.particles_to_c(parts), None,
                                  ct.byref(b))
        return st, lib.lbm_batch_last_error(None).decode()

    def cfgs_of(cs, **over):
        out = []
        for c in cs:
            kw = W.sim_kwargs(c)
            kw.update(over)
            out.append(binding.make_config(c["shape"], **kw))
        return out

    parts = [c["particles"][0] for c in cases]
    st, msg = create(cfgs_of(cases, coupling="MEM_MR", tau=0.875), parts)  # Lambda_- = 1/2
    assert st == binding.LBM_ERR_UNSUPPORTED and "case 0" in msg and "MR" in msg
    st, msg = create(cfgs_of(cases, coupling="NONE"), parts)
    assert st == binding.LBM_ERR_ARG
    cfgs = cfgs_of(cases)
    cfgs[2].storage = binding.STORAGE["f64fx"]
    st, msg = create(cfgs, parts)
    assert st == binding.LBM_ERR_ARG and "case 2" in msg and "storage" in msg
    st, msg = create(cfgs_of(cases, storage="f32"), parts)
    assert st == binding.LBM_ERR_UNSUPPORTED
    big = [dict(p) for p in parts]
    big[1]["diameter"] = 100.0
    st, msg = create(cfgs_of(cases), big)
    assert st == binding.LBM_ERR_ARG and "case 1" in msg
    st, msg = create([], [])
    assert st == binding.LBM_ERR_ARG


# ---- lbm_sweep_noalloc: host-side checks, with no GPU present ------------------------
# These calls carry made-up device addresses.  Without a CUDA device nothing can
# be dereferenced: a call that passes the checks stops at the device lookup
# (LBM_ERR_CUDA).  With a device the same calls could launch kernels on those
# addresses, so the tests only run where there is none.
def _has_cuda():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


no_device = pytest.mark.skipif(_has_cuda(), reason="runs only where no CUDA device exists")


def _noalloc(cfg, parts):
    err = ct.create_string_buffer(256)
    lib = binding.load()
    st = lib.lbm_sweep_noalloc(ct.byref(cfg), ct.c_void_p(0x1000), ct.c_void_p(0x2000),
                               len(parts), binding.particles_to_c(parts),
                               ct.c_void_p(0x3000), None, None, err, len(err))
    return st, err.value.decode()


def _spheres(n, D, L):
    """n spheres of diameter D on a grid of an L^3 periodic box (overlaps allowed:
    only the scratch check is exercised)."""
    return [{"x": (4.0 + 7.0 * (i % 8), 4.0 + 7.0 * (i // 8), L / 2.0), "diameter": D,
             "fixed": 1} for i in range(n)]


@no_device
def test_noalloc_scratch_limit_on_the_host():
    """D = 24 in a 64^3 box: region extent E = ceil(D) + 6 = 30 cells per axis,
    B = ceil(30/32) * ceil(30/2) * 30 = 450 near blocks, so n spheres need
    n^2 * 450 * 6 doubles of force partials: 13 -> 456,300 fit the 524,288 of
    the fixed scratch, 14 -> 529,200 do not.  One sphere of D = 100 in a 128^3
    box needs 106^3 = 1,191,016 geometry-map entries, beyond the 1,048,576,
    while its 4 * 53 * 106 * 6 = 134,832 partials fit."""
    cfg = binding.make_config((64, 64, 64), coupling="PSM_M1B1", tau=0.8)
    st, msg = _noalloc(cfg, _spheres(14, 24.0, 64))
    assert st == binding.LBM_ERR_ARG and "force-partial" in msg and "529200" in msg, msg
    st, msg = _noalloc(cfg, _spheres(13, 24.0, 64))
    assert st == binding.LBM_ERR_CUDA, (st, msg)  # passed every check, then found no device
    cfg = binding.make_config((128, 128, 128), coupling="MEM_CLI", tau=0.8)
    st, msg = _noalloc(cfg, [{"x": (64.0, 64.0, 64.0), "diameter": 100.0, "fixed": 1}])
    assert st == binding.LBM_ERR_ARG and "geometry-map" in msg, msg


@no_device
def test_noalloc_checks_the_configuration_as_lbm_create_does():
    """The allocation-free sweep and lbm_create share their configuration checks:
    a TRT collision needs Lambda > 0 (Eq. (11)), the supersampling at most 40^3,
    finite body forces; MR is refused next to Lambda_- = 1/2."""
    lib = binding.load()
    h = ct.c_void_p()
    bad = [dict(magic=0.0), dict(magic=-0.1), dict(subsample=41), dict(tau=0.5),
           dict(fext=(float("nan"), 0.0, 0.0))]
    for over in bad:
        kw = dict(coupling="PSM_M2B2", tau=0.8)
        kw.update(over)
        cfg = binding.make_config((16, 16, 16), **kw)
        assert lib.lbm_create(ct.byref(cfg), None, ct.byref(h)) == binding.LBM_ERR_ARG, over
        st, msg = _noalloc(cfg, [])
        assert st == binding.LBM_ERR_ARG and "configuration" in msg, (over, msg)
    cfg = binding.make_config((16, 16, 16), coupling="MEM_MR", tau=0.875)
    assert _noalloc(cfg, [])[0] == binding.LBM_ERR_UNSUPPORTED
    cfg = binding.make_config((16, 16, 16), coupling="PSM_M2B2", tau=0.8, storage="f32")
    assert _noalloc(cfg, [])[0] == binding.LBM_ERR_UNSUPPORTED
