"""The C ABI without a GPU: the library builds for sm_103a, loads, exports
every entry point include/pfarna.h declares, its structs match the ctypes
mirrors, and the host-side validation rejects bad arguments."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_1310_4624_gb300 import binding as B
from paper_1310_4624_gb300 import build as cuda_build
from paper_1310_4624_gb300 import synth
from paper_1310_4624_gb300.filter import config_from_workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pfarna.h")


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return B.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pf_[a-z_]+)\s*\(", text)))


def test_header_declares_what_the_binding_wraps():
    assert declared_functions() == sorted(B.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert lib.pf_abi_version() == 5


def test_struct_layout_matches_ctypes(tmp_path):
    exe = str(tmp_path / "probe")
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", exe,
                    os.path.join(ROOT, "tests", "abi_layout_probe.c")], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        struct, field, val = line.split()
        cls = getattr(B, struct)
        if field == "sizeof":
            assert C.sizeof(cls) == int(val), line
        else:
            assert getattr(cls, field).offset == int(val), line


def _cfg(**kw):
    c = config_from_workload(synth.small_rna())
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def test_query_workspace_scales_with_particles(lib):
    a = B.pf_query_workspace([_cfg()], 16)
    b = B.pf_query_workspace([_cfg(Np=4096)], 16)
    assert 0 < a < b
    # 48 bytes of particle state per particle at least (two 20-byte state buffers, ancestors, weights)
    assert b - a >= (4096 - 1024) * 4 * 48 * 0.9
    assert B.pf_query_workspace([_cfg(), _cfg(G=7, Np=333)], 4) > a


@pytest.mark.parametrize("field,value,msg", [
    ("G", 0, "G must be"), ("Np", 0, "Np must be"), ("H", 0, "H and W"), ("patch_radius", 9, "patch_radius"),
    ("mode", 3, "mode"), ("init_kind", 7, "init_kind"), ("sigma_psf", 0.0, "sigma_psf"),
    ("sigma_obs", -1.0, "sigma_obs"), ("sigma_pos", float("nan"), "process noise"), ("ex_ratio", 1.5, "ex_ratio"),
    ("track_id", 1 << 24, "track_id"), ("obs_model", 2, "obs_model"), ("G", 1025, "G must be"),
    ("Np", (1 << 20) + 1, "Np must be"), ("resample_rule", 2, "resample_rule"), ("ess_fraction", 1.5, "ess_fraction"),
    ("ess_fraction", float("nan"), "ess_fraction"), ("send_rule", 2, "send_rule"),
    ("topology", 3, "topology"),
])
def test_invalid_configs_are_rejected_on_the_host(lib, field, value, msg):
    with pytest.raises(B.PFError) as e:
        B.pf_query_workspace([_cfg(**{field: value})], 4)
    assert e.value.status == B.PF_ERR_ARG
    assert msg in str(e.value)
    assert msg in B.pf_last_error(None)


def test_node_ring_needs_node_groups(lib):
    with pytest.raises(B.PFError) as e:
        B.pf_query_workspace([_cfg(topology=B.PF_TOPO_NODE_RING, node_groups=0)], 4)
    assert e.value.status == B.PF_ERR_ARG and "node_groups" in str(e.value)
    assert B.pf_query_workspace([_cfg(topology=B.PF_TOPO_NODE_RING, node_groups=3)], 4) > 0
    assert B.pf_query_workspace([_cfg(node_groups=0)], 4) > 0  # ignored by the other topologies


def test_mixed_patch_radius_and_bad_history_rejected(lib):
    with pytest.raises(B.PFError):
        B.pf_query_workspace([_cfg(), _cfg(patch_radius=4)], 4)
    with pytest.raises(B.PFError):
        B.pf_query_workspace([_cfg()], 0)


def test_init_rejects_bad_workspace_without_touching_the_gpu(lib):
    c = (B.pf_track_config * 1)(_cfg())
    h = C.c_void_p()
    n = B.pf_query_workspace([_cfg()], 4)
    assert lib.pf_init(c, 1, 4, None, n, None, None, C.byref(h)) == B.PF_ERR_ARG
    assert lib.pf_init(c, 1, 4, C.c_void_p(256 * 1000 + 8), n, None, None, C.byref(h)) == B.PF_ERR_WORKSPACE
    assert lib.pf_init(c, 1, 4, C.c_void_p(256 * 1000), n - 1, None, None, C.byref(h)) == B.PF_ERR_WORKSPACE
    user = (B.pf_track_config * 1)(_cfg(init_kind=B.PF_INIT_USER))
    assert lib.pf_init(user, 1, 4, C.c_void_p(256 * 1000), n, None, None, C.byref(h)) == B.PF_ERR_ARG
    assert h.value is None


def test_handle_less_calls_validate(lib):
    assert lib.pf_resample_workspace(0, 5, C.byref(C.c_size_t())) == B.PF_ERR_ARG
    n = C.c_size_t()
    assert lib.pf_resample_workspace(3, 5, C.byref(n)) == B.PF_OK and n.value > 0
    assert lib.pf_resample(None, None, 3, 5, None, None, None, 0, None) == B.PF_ERR_ARG
    assert lib.pf_step(None, None, None) == B.PF_ERR_ARG
    assert lib.pf_estimate(None, None, None) == B.PF_ERR_ARG
    assert lib.pf_step_host(None, None, None, 0, None) == B.PF_ERR_ARG
    assert lib.pf_host_staging_bytes(None, C.byref(n)) == B.PF_ERR_ARG


def test_build_targets_sm103a_only():
    assert cuda_build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library every call raises (no CPU fallback)."""
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B._build, "LIB", str(tmp_path / "libpfarna.so"))
    with pytest.raises(RuntimeError, match="not built"):
        B.load()
    with pytest.raises(RuntimeError, match="not built"):
        B.pf_query_workspace([_cfg()], 4)


def test_product_package_does_not_use_the_oracle():
    """The package (binding, wrapper, kernels) never imports, loads or runs
    anything under oracle/: the oracle is test infrastructure."""
    pkg = os.path.join(ROOT, "paper_1310_4624_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, flags=re.M), f
                assert "pf_oracle" not in text and "liboracle" not in text, f
