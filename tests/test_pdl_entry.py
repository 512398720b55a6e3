"""Source check of the programmatic-dependent-launch rule: every kernel that
the library launches through pdl() (programmatic stream serialization, so
its blocks may start while the previous kernel on the stream finishes) must
call pdl_entry() (griddepcontrol.wait) before anything else, or it could
read or overwrite data the previous kernel has not finished with."""

import glob
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2010_12879_gb300", "csrc")


def _sources():
    return {p: open(p).read() for p in sorted(glob.glob(os.path.join(CSRC, "*.cu")) +
                                              glob.glob(os.path.join(CSRC, "*.cuh")))}


def _matching(s, i):
    depth = 0
    for j in range(i, len(s)):
        if s[j] == "(":
            depth += 1
        elif s[j] == ")":
            depth -= 1
            if depth == 0:
                return j
    raise ValueError("unbalanced parentheses")


def test_every_pdl_kernel_starts_with_pdl_entry():
    src = _sources()
    launched = set()
    for text in src.values():
        launched.update(re.findall(r"\bpdl\(\s*(k_\w+)", text))
    assert len(launched) >= 20, sorted(launched)
    missing = []
    for name in sorted(launched):
        defs = 0
        for text in src.values():
            for m in re.finditer(r"__global__[^;{]*?\b%s\s*\(" % re.escape(name), text):
                close = _matching(text, m.end() - 1)
                brace = text.index("{", close)
                body = text[brace + 1:].lstrip()
                defs += 1
                if not body.startswith("pdl_entry();"):
                    missing.append(name)
        assert defs >= 1, f"no definition of {name}"
    assert not missing, f"kernels launched by pdl() without pdl_entry() first: {missing}"


def test_pdl_attribute_is_switchable_and_off_in_capture():
    """pdl_entry() is harmless in a plain launch (the wait returns at once),
    so a kernel may be launched both ways; this checks that the helper keeps
    the attribute switchable (graph capture turns it off)."""
    text = open(os.path.join(CSRC, "spfd_internal.cuh")).read()
    assert "cudaLaunchAttributeProgrammaticStreamSerialization" in text
    assert "pdl_allowed ? 1 : 0" in text
    graph = open(os.path.join(CSRC, "spfd_graph.cu")).read()
    assert "pdl_allowed = false" in graph
