"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/ccm.h declares; the ctypes binding matches the header."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    """{name: number of parameters} of the CCM_API functions in ccm.h."""
    src = open(os.path.join(ROOT, "include", "ccm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"CCM_API\s+[\w\s\*]+?\b(ccm_\w+)\s*\(([^)]*)\)\s*;", src):
        args = m.group(2).strip()
        out[m.group(1)] = 0 if args in ("", "void") else len(args.split(","))
    return out


@pytest.fixture(scope="module")
def lib():
    from paper_2604_17538_b300 import abi, build
    build.build()
    return abi.lib()


def test_header_declares_the_boundary():
    names = set(_declared())
    for n in ("ccm_create", "ccm_destroy", "ccm_load_geometry", "ccm_free_geometry",
              "ccm_output_size", "ccm_batch_create", "ccm_contacts", "ccm_contacts_backward",
              "ccm_last_error", "ccm_serve_start", "ccm_serve_stop", "ccm_submit", "ccm_poll"):
        assert n in names, n


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_matches_header(lib):
    from paper_2604_17538_b300 import abi
    decl = _declared()
    for name, (_, args) in abi._SIGS.items():
        assert name in decl, f"{name} bound but not declared"
        assert len(args) == decl[name], (name, len(args), decl[name])
    missing = set(decl) - set(abi._SIGS)
    assert not missing, f"declared but not bound: {sorted(missing)}"


def test_no_device_needed_for_defaults(lib):
    from paper_2604_17538_b300 import abi
    p = abi.default_params()
    assert abs(p.tau_sdf - 5e-3) < 1e-9 and p.trace_iters == 3 and p.d_max > 0
    assert lib.ccm_last_error() is not None


def test_serve_config_layout_and_defaults(lib):
    """The ctypes struct mirrors ccm_serve_config: the library's defaults land
    in the right fields (a layout mismatch would scramble them)."""
    from paper_2604_17538_b300 import abi
    c = abi.default_serve_config()
    assert (c.max_wave_pairs, c.max_wave_requests, c.max_queued) == (16384, 1024, 65536)
    assert abs(c.params.tau_sdf - 5e-3) < 1e-9 and c.params.trace_iters == 3
    assert (c.tuning.item_v, c.tuning.item_e, c.tuning.fwd_warps) == (256, 512, 2)
