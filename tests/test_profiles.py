"""The ncu summaries under profiles/ state commands that run committed files
only: every command is a bench.py invocation this bench.py accepts, every
ncu command leaves the clocks alone (--clock-control none), the full-set
captures take one to three launches of one kernel that the library defines,
and no summary names a scratch path or a run of its own making."""
import glob
import os
import re
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*")))
CSRC = os.path.join(ROOT, "paper_1511_01561_gb300", "csrc")


def _command(path):
    with open(path) as f:
        text = f.read()
    m = re.search(r"```\n(.*?)\n```", text, re.S)
    assert m, f"{path}: no command block"
    return text, shlex.split(m.group(1))


def _strip_launch_bounds(src):
    """The source without its __launch_bounds__(...) qualifiers (balanced
    parentheses: the bounds are expressions)."""
    out, i = [], 0
    while True:
        j = src.find("__launch_bounds__", i)
        if j < 0:
            return "".join(out) + src[i:]
        out.append(src[i:j])
        k, depth = src.index("(", j), 0
        while True:
            depth += {"(": 1, ")": -1}.get(src[k], 0)
            k += 1
            if depth == 0:
                break
        i = k


def _global_kernels():
    names = set()
    for src in glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")):
        with open(src) as f:
            names.update(re.findall(r"__global__\s+void\s+(\w+)\s*\(", _strip_launch_bounds(f.read())))
    return names


def test_profiles_exist_as_short_text():
    assert PROFILES
    for p in PROFILES:
        assert p.endswith((".md", ".txt")), p
        assert os.path.getsize(p) < 16 * 1024, p
        name = os.path.basename(p)
        assert not re.search(r"(^|_)r\d\d(_|\.)|round", name), name


@pytest.mark.parametrize("path", PROFILES, ids=[os.path.basename(p) for p in PROFILES])
def test_profile_command_runs_committed_files(path):
    text, argv = _command(path)
    assert "gpurun" not in text and "/root/" not in text and "_work/" not in text
    if argv[0] == "ncu":
        assert "--clock-control" in argv and argv[argv.index("--clock-control") + 1] == "none"
        i = argv.index("python")
        opts, prog = argv[1:i], argv[i + 1:]
        if "--set" in opts:
            # a full-set capture: one kernel, one to three launches
            assert 1 <= int(opts[opts.index("-c") + 1]) <= 3
            pattern = opts[opts.index("-k") + 1]
            assert pattern.startswith("regex:")
            # a mangled name "<kernel>I<template args>E": the kernel is one of the library's
            kernel = re.match(r"regex:(\w+?)I", pattern).group(1)
            assert kernel in _global_kernels(), kernel
        else:
            assert opts[:2] == ["--metrics", "gpu__time_duration.sum"]
    else:
        assert argv[0] == "python"
        prog = argv[1:]
    assert prog[0] == "bench.py" and os.path.exists(os.path.join(ROOT, prog[0]))
    args = bench.parse_args(prog[1:])
    assert args.gpus == 1
