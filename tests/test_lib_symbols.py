"""The C-ABI library builds, loads without a GPU and exports every function that
include/*.h declares (no compute calls)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*\**\s+\**(mdwf_[A-Za-z0-9_]+)\s*\(",
                            src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_1810_01609_gb300", "lib", "libmdwf.so"))
    names = _declared()
    assert len(names) >= 20, names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_argument_validation():
    """Host logic that needs no GPU: parameter validation and status strings."""
    import __graft_entry__
    __graft_entry__.build()
    import paper_1810_01609_gb300 as m
    assert m.strerror(m.MDWF_ERR_NOT_SU3) == "gauge link not in SU(3)"
    p = m.mdwf_default_params()
    assert (p.Ls, p.b5, p.c5, p.M5) == (8, 1.5, 0.5, 1.3)
    for bad in ({"dims": (3, 4, 4, 4)}, {"Ls": 1}, {"Ls": 40}, {"gauge_recon": 9}):
        q = m.mdwf_default_params()
        for k, v in bad.items():
            if k == "dims":
                for i in range(4):
                    q.dims[i] = v[i]
            else:
                setattr(q, k, v)
        try:
            m.mdwf_create(q)
            raise AssertionError("accepted %r" % bad)
        except m.MdwfError as e:
            assert e.code == m.MDWF_ERR_ARG
    assert m.mdwf_default_params().f64_emulation == 1
    ctx = m.mdwf_create(m.mdwf_default_params())
    assert m.mdwf_field_bytes(ctx, 2, 1) > m.mdwf_field_bytes(ctx, 3, 1)
    # emulated FP64 uses the FP64 storage layout
    assert m.mdwf_field_bytes(ctx, m.PRECS["f64e"], 1) == m.mdwf_field_bytes(ctx, 0, 1)
    # the one-call propagator rejects missing buffers before touching the device
    infos = (m.mdwf_solve_info * 1)()
    sp = m.mdwf_default_solve_params()
    code = m.load().mdwf_propagator(ctx, 1, None, None, m.MDWF_HOST, ctypes.byref(sp), infos, None)
    assert code == m.MDWF_ERR_ARG
    try:
        m.mdwf_field_bytes(ctx, 7, 1)
        raise AssertionError
    except m.MdwfError as e:
        assert e.code == m.MDWF_ERR_ARG
    m.mdwf_destroy(ctx)


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C compiler's sizes and offsets."""
    import subprocess
    import paper_1810_01609_gb300._lib as L
    structs = {"mdwf_params": L.mdwf_params, "mdwf_solve_params": L.mdwf_solve_params,
               "mdwf_solve_info": L.mdwf_solve_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mdwf.h"', "int main(void) {"]
    for sname, cls in structs.items():
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (sname, sname))
        for fname, _ in cls._fields_:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (sname, fname, sname, fname))
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for sname, cls in structs.items():
        assert int(got[sname]) == ctypes.sizeof(cls), sname
        for fname, _ in cls._fields_:
            assert int(got["%s.%s" % (sname, fname)]) == getattr(cls, fname).offset, (sname, fname)


def test_fh_effective_coupling_matches_oracle():
    """Host-side C function of the library against the oracle's estimator (no GPU)."""
    import __graft_entry__
    __graft_entry__.build()
    import numpy as np
    import paper_1810_01609_gb300 as m
    from oracle import hadron
    rng = np.random.default_rng(3)
    c2 = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    c3 = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    got = m.mdwf_fh_effective_coupling(c2, c3)
    assert np.max(np.abs(got - hadron.fh_effective_coupling(c2, c3))) <= 1e-13 * np.max(np.abs(got))
    c2[5] = 0.0
    try:
        m.mdwf_fh_effective_coupling(c2, c3)
        raise AssertionError("accepted C(t) = 0")
    except m.MdwfError as e:
        assert e.code == m.MDWF_ERR_ARG
