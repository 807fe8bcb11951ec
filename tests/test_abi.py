"""CPU checks of the C-ABI library: it builds, loads, and exports every
function include/idos.h declares (no compute call: there may be no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "idos.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(idos_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_boundary():
    names = declared_functions()
    for must in ("idos_create_model", "idos_sample_level", "idos_eval_idos", "idos_mlmc_estimate",
                 "idos_get_level_stats", "idos_destroy_model", "idos_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1611_09784_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_loads_and_status_strings():
    import paper_1611_09784_gb300 as pkg
    pkg.load_library()
    assert pkg.status_string(0) == "ok"
    assert pkg.status_string(-1) == "invalid argument"
    assert pkg.status_string(-7) == "no sm_103 device"


def test_create_model_rejects_bad_descriptors_without_gpu():
    """Descriptor validation runs before any device call."""
    import paper_1611_09784_gb300 as pkg
    base = dict(levels=[(4, 6), (8, 3)], p=0.05)
    for bad in (dict(levels=[(4, 6), (6, 3)]), dict(p=1.5), dict(n_E=1), dict(delta=0.0),
                dict(e_min=1.0, e_max=0.0), dict(levels=[(65, 1)])):
        cfg = dict(base)
        cfg.update(bad)
        with pytest.raises(pkg.IdosError) as ei:
            pkg.create_model(cfg)
        assert ei.value.status == -1
    with pytest.raises(pkg.IdosError) as ei:
        pkg.create_model(dict(base, kind="tmdc"))
    assert ei.value.status in (-6, -7)


def test_no_oracle_import_in_product():
    """The product package never imports the oracle."""
    pkgdir = os.path.join(ROOT, "paper_1611_09784_gb300")
    for dp, _, fs in os.walk(pkgdir):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_dos_from_idos_matches_oracle():
    """idos_dos_from_idos is host arithmetic (no device): central differences
    of the IDoS against the oracle's."""
    import numpy as np
    import paper_1611_09784_gb300 as pkg
    from oracle import idos as oidos
    rng = np.random.default_rng(3)
    Q = np.cumsum(rng.random(201)) * 1e-3
    got = pkg.dos_from_idos(Q, -9.0, 9.0)
    ref = oidos.dos_from_idos(Q, -9.0, 9.0)
    assert np.allclose(got, ref, rtol=1e-14, atol=0)
    with pytest.raises(pkg.IdosError):
        pkg.dos_from_idos(Q[:1], -9.0, 9.0)


def test_struct_layouts_match_binding(tmp_path):
    """Every public struct of include/idos.h has the binding's field names,
    offsets and size (compiled with the host C compiler)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    from paper_1611_09784_gb300 import binding as b
    structs = {"idos_model_desc": b.ModelDesc, "idos_mlmc_opts": b.MlmcOpts, "idos_estimate": b.Estimate,
               "idos_tuning": b.Tuning}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "idos.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} . %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    for line in out.splitlines():
        cname, fname, value = line.split()
        cls = structs[cname]
        want = ctypes.sizeof(cls) if fname == "." else getattr(cls, fname).offset
        assert int(value) == want, (cname, fname, int(value), want)
