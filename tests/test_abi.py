"""The C-ABI library loads, exports every declared symbol, and validates
descriptions on the host (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2310_04676_gb300 import sg, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(sg.LIB_PATH):
        from paper_2310_04676_gb300 import build
        build.build()
    return sg.load_library()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(sg_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_plan_counts_and_obs_dim(lib):
    kinds = W.mixed_kinds(1000, W.C3_FRACTIONS)
    d = W.make_desc(kinds)
    info = sg.plan(d)
    assert info["obs_dim"] == 54
    n4 = kinds.count("4R")
    n7 = kinds.count("7R")
    n7p = kinds.count("7P")
    nb = kinds.count("14B")
    assert info["class_slots"] == [n7 + 2 * nb, n7p, 0, n4]
    assert info["num_chains"] == n4 + n7 + n7p + 2 * nb
    assert info["num_slots"] % 32 == 0


def test_plan_three_arm_groups(lib):
    d = W.make_desc(["21T"] * 5 + ["7R"] * 3)
    info = sg.plan(d)
    assert info["obs_dim"] == 3 * 21 + 18
    assert info["class_slots"] == [3, 15, 0, 0]
    assert info["num_chains"] == 18


def test_plan_generic_class_and_path_obs(lib):
    from tests.helpers import chain_desc
    d = chain_desc([([0, 1, 0], [0, 2, 1])], E=5)
    info = sg.plan(d)
    assert info["class_slots"] == [0, 0, 5, 0]
    dp = W.make_desc(["7R"] * 3, task=1, path_len=8)
    assert sg.plan(dp)["obs_dim"] == 30


@pytest.mark.parametrize("mutate,code", [
    (lambda d: d.__setitem__("num_envs", 0), sg.SG_ERR_INVALID_ARG),
    (lambda d: d["env_num_chains"].__setitem__(0, 3), sg.SG_ERR_INVALID_ARG),
    (lambda d: d["chain_num_joints"].__setitem__((0, 0), 8), sg.SG_ERR_INVALID_ARG),
    (lambda d: d["joint_axis"].__setitem__((0, 1), 5), sg.SG_ERR_INVALID_ARG),
    (lambda d: d["link_mass"].__setitem__((0, 2), 0.0), sg.SG_ERR_INVALID_ARG),
    (lambda d: d["link_len"].__setitem__((0, 2), np.nan), sg.SG_ERR_INVALID_ARG),
    (lambda d: d["kp"].__setitem__((0, 2), -1.0), sg.SG_ERR_INVALID_ARG),
    (lambda d: (d["joint_type"].__setitem__((0, 1), 1), d["joint_axis"].__setitem__((0, 1), 1)),
     sg.SG_ERR_UNSUPPORTED),
    (lambda d: d.__setitem__("episode_len", 0), sg.SG_ERR_INVALID_ARG),
    (lambda d: d.__setitem__("task", 7), sg.SG_ERR_INVALID_ARG),
    (lambda d: d.__setitem__("joint_drive", np.full((2, 7), 3, np.int32)), sg.SG_ERR_INVALID_ARG),
    (lambda d: (d.__setitem__("task", 2), d.__setitem__("track_sigma", 0.0)), sg.SG_ERR_INVALID_ARG),
])
def test_plan_rejects_bad_descriptions(lib, mutate, code):
    d = W.make_desc(["7R", "4R"])
    d = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in d.items()}
    mutate(d)
    with pytest.raises(sg.SgError) as ei:
        sg.plan(d)
    assert ei.value.status == code


def test_path_task_rejects_two_arm_envs(lib):
    d = W.make_desc(["7R", "14B"])
    d["task"] = 1
    d["path_len"] = 8
    d["path"] = np.zeros((2, 8, 3), np.float32)
    with pytest.raises(sg.SgError) as ei:
        sg.plan(d)
    assert ei.value.status == sg.SG_ERR_UNSUPPORTED


def test_path_task_inputs_are_validated(lib):
    d = W.make_desc(["7R"] * 3, task=1, path_len=8)
    sg.plan(d)                                             # control points only: fine
    both = dict(d, path=np.zeros((3, 8, 3), np.float32))
    short = dict(d, path_ctrl_len=1, path_ctrl=d["path_ctrl"][:, :1].copy())
    bad = dict(d, path_ctrl=d["path_ctrl"].copy())
    bad["path_ctrl"][1, 3, 2] = np.inf
    few = dict(d, path_len=3)
    for dd in (both, short, bad, few):
        with pytest.raises(sg.SgError) as ei:
            sg.plan(dd)
        assert ei.value.status == sg.SG_ERR_INVALID_ARG
    long_ = dict(d, path_ctrl_len=65, path_ctrl=np.zeros((3, 65, 3), np.float32))
    with pytest.raises(sg.SgError):
        sg.plan(long_)


def test_null_context_calls_are_rejected(lib):
    assert lib.sg_step(None, None, ctypes.c_float(0.01), 1, None, None, None) == sg.SG_ERR_INVALID_ARG
    assert lib.sg_reset(None, None) == sg.SG_ERR_INVALID_ARG
    assert lib.sg_obs_dim(None) == 0
    lib.sg_destroy(None)


# ---- device ownership of a context ------------------------------------------
DEVCHECK_DRIVER = r'''
#include "sg_devcheck.h"
#include <cstring>
// a stand-in for cudaGetDevice: returns `err`, reports device `cur`
extern "C" int check(int owner, int cur, int err, char* msg, int len) {
  std::string m;
  const sg_status st = sg::check_device(
      owner, [&](int* d) { *d = cur; return err; }, "sg_step", &m);
  std::strncpy(msg, m.c_str(), (size_t)len - 1);
  msg[len - 1] = 0;
  return (int)st;
}
'''


def test_device_check_reports_a_mismatched_current_device(tmp_path):
    """The check every entry point runs before enqueuing work, compiled for
    the host against a stand-in device query: the owner's device current ->
    SG_OK; another device current -> SG_ERR_INVALID_ARG naming both devices
    (the call then enqueues nothing); a failing query -> SG_ERR_CUDA."""
    import shutil
    import subprocess
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("needs a host C++ compiler")
    src = tmp_path / "devcheck.cpp"
    src.write_text(DEVCHECK_DRIVER)
    so = tmp_path / "devcheck.so"
    subprocess.run([cxx, "-std=c++17", "-shared", "-fPIC", "-O1",
                    "-I" + os.path.join(ROOT, "include"),
                    "-I" + os.path.join(ROOT, "paper_2310_04676_gb300", "csrc"),
                    str(src), "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    buf = ctypes.create_string_buffer(256)
    assert lib.check(1, 1, 0, buf, 256) == sg.SG_OK and buf.value == b""
    assert lib.check(1, 0, 0, buf, 256) == sg.SG_ERR_INVALID_ARG
    assert b"device 1" in buf.value and b"device 0 is current" in buf.value
    assert b"sg_step" in buf.value
    assert lib.check(0, 3, 0, buf, 256) == sg.SG_ERR_INVALID_ARG
    assert lib.check(2, 2, 100, buf, 256) == sg.SG_ERR_CUDA


def _extern_c_functions(path):
    """{name: body} of the functions of a source file that take a context."""
    text = open(path).read()
    out = {}
    for m in re.finditer(r"\n(?:extern \"C\" )?(?:sg_status|void|int32_t|int64_t|const char\*) "
                         r"(sg_\w+)\(([^)]*)\)\s*\{", text):
        if "sg_ctx" not in m.group(2) and "sg_ppo*" not in m.group(2):
            continue
        depth, i = 1, m.end()
        while depth:
            depth += {"{": 1, "}": -1}.get(text[i], 0)
            i += 1
        out[m.group(1)] = (m.group(2), text[m.end():i])
    return out


# calls that touch no device state (host-side settings and queries), and the
# two destructors, which switch to the owning device instead of refusing
NO_DEVICE_WORK = {"sg_set_stream", "sg_set_launch", "sg_get_launch", "sg_set_host_io",
                  "sg_debug_set_fault", "sg_obs_dim", "sg_num_envs", "sg_max_joints",
                  "sg_last_error", "sg_device", "sg_ppo_num_params", "sg_get_packing"}
SWITCHING = {"sg_destroy", "sg_ppo_destroy"}


def test_every_entry_point_checks_the_device():
    """Every exported call that takes a context and enqueues work or reads
    device state runs the device check before anything else reaches the
    device; the destructors release on the owning device."""
    csrc = os.path.join(ROOT, "paper_2310_04676_gb300", "csrc")
    seen = {}
    for f in ("sg_api.cu", "sg_ppo.cu", "sg_noalloc.cu"):
        seen.update(_extern_c_functions(os.path.join(csrc, f)))
    declared = set(declared_functions())
    assert {"sg_step", "sg_rollout", "sg_ppo_update", "sg_diff_track_noalloc"} <= set(seen)
    for name, (params, body) in seen.items():
        if name not in declared or name in NO_DEVICE_WORK:
            continue
        if name in SWITCHING:
            assert "cudaSetDevice" in body, name
            continue
        if name == "sg_create":               # records the owning device
            assert "cudaGetDevice(&c->device)" in body
            continue
        first_cuda = re.search(r"\bcuda\w+\(|launch_|run_rollout|snapshot\(|pipelined_", body)
        check = re.search(r"SG_CHECK_DEVICE|SG_PPO_CHECK_DEVICE|context_check_device", body)
        assert check, "%s does not check the device" % name
        assert first_cuda is None or check.start() < first_cuda.start(), name
