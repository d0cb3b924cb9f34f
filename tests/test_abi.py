"""The C-ABI library loads and exports every entry point that include/eacg.h declares
(no compute call: this runs without a GPU)."""
import ctypes
import json
import os
import re

from tests.conftest import ROOT, ensure_library


def _declared():
    src = open(os.path.join(ROOT, "include", "eacg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eacg_[a-z_A-Z]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("eacg_create_system", "eacg_apply_H", "eacg_density", "eacg_step", "eacg_solve"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(ensure_library())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params_are_the_paper_constants():
    ensure_library()
    import paper_2503_16225_gb300 as E
    p = E.eacg_default_params()
    c = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    for key in ("delta", "sigma", "gamma", "eps", "mu", "fom_rtol"):
        assert getattr(p, key) == c[key]["value"], key


def test_bytes_required_and_model_validation_on_host():
    ensure_library()
    import synth
    import paper_2503_16225_gb300 as E
    n, per = E.eacg_bytes_required(synth.config_diamond(2))
    assert n > 0 and per > 0
    bad = dict(synth.config_two_atom(1))
    bad["N"] = 7   # not a supported FFT size
    assert E.eacg_bytes_required(bad)[0] == 0
    # band limits: the 64-atom supercell (128 bands) is accepted, 1025 bands are not
    assert E.eacg_bytes_required(synth.config_diamond_supercell(2))[0] > 0
    big = dict(synth.config_diamond(2, kgrid=(1, 1, 1)))
    big["nbands"] = E.EACG_MAX_BANDS + 1
    assert E.eacg_bytes_required(big)[0] == 0


def test_binding_band_limits_match_the_header():
    ensure_library()
    import paper_2503_16225_gb300 as E
    src = open(os.path.join(ROOT, "include", "eacg.h")).read()
    for name in ("EACG_MAX_BANDS", "EACG_MAX_BANDS_DENSE"):
        val = int(re.search(rf"#define {name} (\d+)", src).group(1))
        assert getattr(E, name) == val, name


def _header_struct_fields(name):
    """Field names of a typedef struct { ... } name; in include/eacg.h, in order."""
    src = open(os.path.join(ROOT, "include", "eacg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    end = re.search(r"\}\s*" + name + ";", src).start()
    body = src[src.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        decl = re.sub(r"\[[^\]]*\]", "", decl)          # array extents
        for part in decl.split(","):                       # the declared name ends each part
            fields.append(re.findall(r"[A-Za-z_]\w*", part)[-1])
    return fields


def test_binding_structs_match_the_header_layout():
    """The ctypes mirrors of the ABI structs list the header's fields in the header's order
    (a mismatch would shift every later field silently)."""
    ensure_library()
    import paper_2503_16225_gb300 as E
    for cname, py in (("eacg_model", E.EacgModel), ("eacg_params", E.EacgParams),
                      ("eacg_step_info", E.EacgStepInfo), ("eacg_result", E.EacgResult),
                      ("eacg_kernel_stat", E.EacgKernelStat)):
        assert _header_struct_fields(cname) == [f[0] for f in py._fields_], cname


def test_binding_argument_counts_match_the_header():
    """Every entry point the binding declares takes as many arguments as its header prototype."""
    lib = ctypes.CDLL(ensure_library())
    import paper_2503_16225_gb300 as E
    src = open(os.path.join(ROOT, "include", "eacg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    checked = 0
    for name, args in re.findall(r"\b(eacg_[A-Za-z_0-9]+)\s*\(([^)]*)\)\s*;", src, flags=re.S):
        fn = getattr(E.lib, name, None)
        if fn is None or fn.argtypes is None:
            continue
        n = 0 if args.strip() in ("", "void") else len(args.split(","))
        assert len(fn.argtypes) == n, name
        checked += 1
    assert checked >= 20 and lib is not None
