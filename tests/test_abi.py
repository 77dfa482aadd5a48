"""CPU checks of the C ABI: the library builds, loads and exports every entry
point the header declares, and the ctypes structures match the C layout."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rot_vote.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rot_vote_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_11547_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_exports_every_declared_entry_point(lib):
    names = _declared()
    assert "rot_vote_solve" in names and "rot_vote_submit" in names and "rot_vote_poll" in names
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (rot_vote_\w+)", out))
    assert set(names) <= exported


def test_binding_names_match_header():
    from paper_2506_11547_gb300 import rot_vote as rv
    assert set(rv.EXPORTS) <= set(_declared())


def test_struct_layout_matches_c():
    from paper_2506_11547_gb300 import rot_vote as rv
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "rot_vote.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(rot_vote_config), sizeof(rot_vote_problem), sizeof(rot_vote_result));
  printf("%zu %zu %zu %zu\n", offsetof(rot_vote_result, status), offsetof(rot_vote_result, ms_gpu),
         offsetof(rot_vote_config, cuda_stream), offsetof(rot_vote_problem, delta));
  printf("%zu\n", offsetof(rot_vote_config, chart));
  printf("%zu %zu %zu %zu\n", sizeof(rot_vote_pose_problem), sizeof(rot_vote_pose_result),
         offsetof(rot_vote_pose_problem, pairs_cap), offsetof(rot_vote_pose_result, status));
  printf("%zu %zu %zu %zu\n", sizeof(rot_vote_peak), offsetof(rot_vote_alg1_problem, peak_out),
         offsetof(rot_vote_alg1_result, npeaks), offsetof(rot_vote_alg1_result, peak_threshold));
  printf("%zu %zu %zu %zu %zu\n", sizeof(rot_vote_alg1_problem), sizeof(rot_vote_alg1_result),
         offsetof(rot_vote_alg1_problem, accumulator), offsetof(rot_vote_alg1_result, samples_cast),
         offsetof(rot_vote_alg1_result, ms_gpu));
  printf("%zu %zu\n", offsetof(rot_vote_alg1_result, vote_path), offsetof(rot_vote_alg1_result, wrapped_words));
  printf("%zu %zu\n", sizeof(rot_vote_stage), offsetof(rot_vote_stage, kernels));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = list(map(int, out))
    assert sizes[0] == ctypes.sizeof(rv.rot_vote_config)
    assert sizes[1] == ctypes.sizeof(rv.rot_vote_problem)
    assert sizes[2] == ctypes.sizeof(rv.rot_vote_result)
    assert sizes[3] == rv.rot_vote_result.status.offset
    assert sizes[4] == rv.rot_vote_result.ms_gpu.offset
    assert sizes[5] == rv.rot_vote_config.cuda_stream.offset
    assert sizes[6] == rv.rot_vote_problem.delta.offset
    assert sizes[7] == rv.rot_vote_config.chart.offset
    assert sizes[8:12] == [ctypes.sizeof(rv.rot_vote_pose_problem), ctypes.sizeof(rv.rot_vote_pose_result),
                           rv.rot_vote_pose_problem.pairs_cap.offset, rv.rot_vote_pose_result.status.offset]
    sizes = sizes[:8] + sizes[12:]
    assert sizes[8] == ctypes.sizeof(rv.rot_vote_peak)
    assert sizes[9] == rv.rot_vote_alg1_problem.peak_out.offset
    assert sizes[10] == rv.rot_vote_alg1_result.npeaks.offset
    assert sizes[11] == rv.rot_vote_alg1_result.peak_threshold.offset
    assert sizes[12] == ctypes.sizeof(rv.rot_vote_alg1_problem)
    assert sizes[13] == ctypes.sizeof(rv.rot_vote_alg1_result)
    assert sizes[14] == rv.rot_vote_alg1_problem.accumulator.offset
    assert sizes[15] == rv.rot_vote_alg1_result.samples_cast.offset
    assert sizes[16] == rv.rot_vote_alg1_result.ms_gpu.offset
    assert sizes[17:19] == [rv.rot_vote_alg1_result.vote_path.offset, rv.rot_vote_alg1_result.wrapped_words.offset]
    assert sizes[19:21] == [ctypes.sizeof(rv.rot_vote_stage), rv.rot_vote_stage.kernels.offset]


def test_missing_library_fails_loudly(tmp_path):
    from paper_2506_11547_gb300 import rot_vote as rv
    with pytest.raises(RuntimeError):
        rv._lib = None
        try:
            rv.load(str(tmp_path / "nope.so"))
        finally:
            rv._lib = None
