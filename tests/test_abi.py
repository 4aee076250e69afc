"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/mdas.h declares.  No compute calls here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "mdas.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mdas_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("mdas_create_system", "mdas_forces", "mdas_md_steps", "mdas_swap_trials",
              "mdas_alchemical_move", "mdas_energy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2005_08348_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2005_08348_gb300 import mdas
    assert sorted(mdas.EXPORTS) == declared()


def test_status_strings_without_gpu():
    from paper_2005_08348_gb300 import mdas
    lib = mdas.lib()
    assert lib.mdas_status_string(0) == b"ok"
    assert lib.mdas_status_string(4) == b"unstable state"


def test_create_rejects_bad_arguments_without_touching_the_gpu():
    """Argument validation happens on the host before any CUDA call."""
    from paper_2005_08348_gb300 import mdas
    lib = mdas.lib()
    d = mdas.Desc()
    out = ctypes.c_void_p()
    assert lib.mdas_create_system(ctypes.byref(d), ctypes.byref(out)) == 1
    assert b"sizes" in lib.mdas_last_error(None)
    assert lib.mdas_create_system(None, ctypes.byref(out)) == 1


def test_tune_list_skin_rejects_bad_arguments_without_touching_the_gpu():
    from paper_2005_08348_gb300 import mdas
    lib = mdas.lib()
    d = mdas.Desc()
    arr = (ctypes.POINTER(mdas.Desc) * 1)(ctypes.pointer(d))
    skins = (ctypes.c_double * 2)(0.3, -0.1)
    us = (ctypes.c_double * 2)()
    best = ctypes.c_double()
    assert lib.mdas_tune_list_skin(arr, 1, skins, 2, 10, 0, 1, us, ctypes.byref(best)) == 1
    assert b"candidate" in lib.mdas_last_error(None)
    assert lib.mdas_tune_list_skin(arr, 0, skins, 1, 10, 0, 1, us, ctypes.byref(best)) == 1
    assert lib.mdas_tune_list_skin(arr, 1, skins, 1, 0, 0, 1, us, ctypes.byref(best)) == 1


def test_no_cpu_fallback_in_the_product_path():
    pkg = os.path.join(ROOT, "paper_2005_08348_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            txt = open(os.path.join(pkg, f)).read()
            assert "import oracle" not in txt and "from oracle" not in txt, f


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes mirror of a header struct has the header's size and field
    offsets (a C program compiled against include/mdas.h prints them)."""
    import ctypes as C
    import shutil
    import subprocess
    from paper_2005_08348_gb300 import mdas
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    trial_names = {"null": "null_trial"}
    pairs = [(mdas.Desc, "mdas_system_desc"), (mdas.EnergyTerms, "mdas_energy_terms"),
             (mdas.SwapStats, "mdas_swap_stats"), (mdas.MoveResult, "mdas_move_result"),
             (mdas.StateView, "mdas_state_view"), (mdas.Counters, "mdas_counters"),
             (mdas.Job, "mdas_job"), (mdas.JobResult, "mdas_job_result")]
    lines, want = [], []
    for py, cname in pairs:
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        want.append(C.sizeof(py))
        for f in py._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {f[0]}));')
            want.append(getattr(py, f[0]).offset)
    lines.append('printf("%zu\\n", sizeof(mdas_trial_record));')
    want.append(mdas.TRIAL_DTYPE.itemsize)
    for name in mdas.TRIAL_DTYPE.names:
        lines.append(f'printf("%zu\\n", offsetof(mdas_trial_record, {trial_names.get(name, name)}));')
        want.append(mdas.TRIAL_DTYPE.fields[name][1])
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"mdas.h\"\nint main(void) {\n"
                   + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == want


def test_footprint_counts_the_pressure_coupling_grids_without_a_gpu():
    """A pressure-coupled system sizes its cell grids for a box that may
    shrink, so its lists hold more entries per bead; the admission estimate
    (host arithmetic only) follows the same sizing."""
    from paper_2005_08348_gb300 import mdas, synth
    m = synth.mcmd_small()
    nvt = mdas.footprint(m)
    npt = mdas.footprint(m, pcouple=dict(box_margin=0.05))
    wide = mdas.footprint(m, pcouple=dict(box_margin=0.2))
    assert nvt < npt < wide
    assert mdas.footprint(m, pcouple=None) == nvt


def test_shape_path_and_state_calls_reject_bad_arguments_without_touching_the_gpu():
    """The step-shape, trial-path, packed-state and batch-tuner calls check
    their arguments on the host first (MDAS_ERR_INVALID_ARG, no CUDA call)."""
    from paper_2005_08348_gb300 import mdas
    lib = mdas.lib()
    assert lib.mdas_set_list_lanes(None, 2) == 1
    assert lib.mdas_set_trial_path(None, 0) == 1
    assert lib.mdas_get_state_packed(None, None, None, None) == 1
    assert lib.mdas_set_state_packed(None, None, None, None) == 1
    d = mdas.Desc()
    arr = (ctypes.POINTER(mdas.Desc) * 1)(ctypes.pointer(d))
    skins = (ctypes.c_double * 1)(0.3)
    waves = (ctypes.c_int64 * 1)(0)
    lanes = (ctypes.c_int32 * 2)(4, 3)                    # 3 lanes per bead does not exist
    us = (ctypes.c_double * 4)()
    best, part, wave, lane = ctypes.c_double(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
    assert lib.mdas_tune_batch(arr, 1, skins, 1, waves, 1, lanes, 2, 10, 0, 1, us, ctypes.byref(best),
                               ctypes.byref(part), ctypes.byref(wave), ctypes.byref(lane)) == 1
    assert b"lanes" in lib.mdas_last_error(None)
    assert lib.mdas_tune_batch(arr, 1, skins, 1, waves, 1, lanes, 0, 10, 0, 1, us, ctypes.byref(best),
                               ctypes.byref(part), ctypes.byref(wave), ctypes.byref(lane)) == 1
