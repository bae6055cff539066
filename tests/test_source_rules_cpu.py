"""Source rules of the CUDA library and of the committed profile commands (CPU only, text checks).

* Every mbarrier wait is bounded: the only ``mbarrier.try_wait`` is the one inside ``tc.cuh``'s
  ``mbar_try_wait``, whose only caller is ``mbar_wait`` (a counted loop that records a status code
  and returns false when the count runs out).  No kernel spins on an mbarrier any other way.
* No device code stops a kernel by faulting: no ``__trap``, no PTX ``trap``, no device ``assert``.
* Every ``ncu`` command in ``profiles/`` leaves the GPU clocks alone (``--clock-control none``).
* No committed code changes a GPU setting through ``nvidia-smi`` (clocks, power, persistence,
  compute mode, reset).
"""

import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1905_07311_gb300", "csrc")


def _sources():
    files = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")))
    assert files
    return {os.path.basename(f): open(f).read() for f in files}


def _strip_comments(text):
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.sub(r"//[^\n]*", "", text)


def test_mbarrier_waits_are_bounded():
    src = {k: _strip_comments(v) for k, v in _sources().items()}
    hits = {k: len(re.findall(r"mbarrier\.(try_wait|test_wait)", v)) for k, v in src.items()}
    assert {k: n for k, n in hits.items() if n} == {"tc.cuh": 1}
    callers = {k: len(re.findall(r"\bmbar_try_wait\s*\(", v)) for k, v in src.items()}
    # the definition and the one call inside mbar_wait
    assert {k: n for k, n in callers.items() if n} == {"tc.cuh": 2}
    tc = src["tc.cuh"]
    body = tc[tc.index("bool mbar_wait("):]
    body = body[:body.index("\n}\n")]
    assert re.search(r"for \(uint32_t it = 0; it < limit; \+\+it\)", body)
    assert "mbar_try_wait(bar, parity)" in body and "return false;" in body


def test_no_device_code_faults_on_purpose():
    for name, text in _sources().items():
        code = _strip_comments(text)
        assert "__trap" not in code, name
        assert not re.search(r"\btrap\s*;", code), name
        assert not re.search(r"(?<![\w.])assert\s*\(", code), name


def test_profile_commands_leave_the_clocks_alone():
    found = 0
    for path in glob.glob(os.path.join(ROOT, "profiles", "*")):
        lines = open(path).read().replace("\\\n", " ").splitlines()
        for line in lines:
            # a command: ncu followed by its options (reading a saved report, ncu -i, runs nothing)
            if re.search(r"(^|[;&|(]\s*|\s)ncu\s+--?[a-z]", line) and not re.search(r"ncu\s+-i\s", line):
                found += 1
                assert "--clock-control none" in line, (os.path.basename(path), line)
    assert found > 0


def test_no_gpu_setting_is_changed():
    setters = re.compile(r"nvidia-smi[^\n]*\s(-lgc|-lmc|-rgc|-rmc|-ac|-rac|-pl|-pm|-c|-r|--lock-gpu-clocks|"
                         r"--lock-memory-clocks|--reset-gpu-clocks|--power-limit|--persistence-mode|"
                         r"--compute-mode|--gpu-reset)\b")
    paths = [os.path.join(ROOT, "bench.py"), os.path.join(ROOT, "__graft_entry__.py")]
    paths += glob.glob(os.path.join(ROOT, "paper_1905_07311_gb300", "*.py"))
    paths += glob.glob(os.path.join(CSRC, "*"))
    paths += glob.glob(os.path.join(ROOT, "tests", "*.py"))
    paths += glob.glob(os.path.join(ROOT, "profiles", "*"))
    me = os.path.abspath(__file__)
    for p in paths:
        if os.path.abspath(p) == me or not os.path.isfile(p):
            continue
        assert not setters.search(open(p, errors="replace").read()), p
