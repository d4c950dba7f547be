"""Host-side checks of the C-ABI library (no GPU needed, no compute calls).

* the shared library loads and exports every function declared in include/*.h;
* the host-only calls (decomposition, workspace sizing) agree with the plain
  definitions in the oracle.
"""
import ctypes
import glob
import os
import re

import pytest

import paper_2102_12416_gb300 as jg
from paper_2102_12416_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return jg.load()


def _declared_functions():
    names = set()
    for path in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(path).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.add(name)
    return names


def test_header_symbols_exported(lib):
    names = _declared_functions()
    assert {"jacobi_create", "jacobi_step", "jacobi_residual", "channel_open", "channel_send",
            "channel_recv"} <= names
    so = ctypes.CDLL(_build.LIB)
    missing = [n for n in sorted(names) if not hasattr(so, n)]
    assert not missing, f"declared but not exported: {missing}"
    # and the binding wraps each one under the same name
    unwrapped = [n for n in sorted(names) if not hasattr(jg, n)]
    assert not unwrapped, f"declared but not in the Python binding: {unwrapped}"


@pytest.mark.parametrize("grid,n", [((64, 64, 64), 8), ((512, 512, 512), 512), ((96, 96, 96), 6),
                                    ((1024, 64, 64), 8), ((1536, 768, 512), 6), ((45, 37, 29), 105),
                                    ((17, 5, 3), 12), ((768, 768, 768), 1728), ((7, 11, 13), 1)])
def test_decompose_matches_oracle(lib, oracle_mod, grid, n):
    assert jg.jacobi_decompose(grid, n) == oracle_mod.decompose(grid, n)


def test_decompose_large_sizes(lib):
    # the largest accepted sizes: a cube splits evenly (the surface sum needs
    # more than 64 bits here), and a prime count can only go along one axis
    n = 1 << 30
    assert jg.jacobi_decompose((n, n, n), n) == (1024, 1024, 1024)
    assert jg.jacobi_decompose((n, 2, 2), 1_000_003) == (1_000_003, 1, 1)
    with pytest.raises(jg.JacobiError):
        jg.jacobi_decompose((n + 1, 2, 2), 2)
    with pytest.raises(jg.JacobiError):
        jg.jacobi_decompose((8, 8, 8), n + 1)


def test_decompose_rejects_impossible(lib):
    with pytest.raises(jg.JacobiError) as e:
        jg.jacobi_decompose((2, 2, 2), 27)
    assert e.value.code == jg.JACOBI_EINVAL


def test_strerror(lib):
    assert lib.jacobi_strerror(jg.JACOBI_ETIMEDOUT) == b"device wait timed out"


def test_workspace_bytes_scale(lib):
    small = jg.jacobi_workspace_bytes((64, 64, 64), ("count", (2, 2, 2)), "f64")
    big = jg.jacobi_workspace_bytes((512, 512, 512), ("count", (8, 8, 8)), "f64")
    f32 = jg.jacobi_workspace_bytes((512, 512, 512), ("count", (8, 8, 8)), "f32")
    # two state copies dominate: 2 * 8 B * 512^3 = 2.1 GB
    assert 2 * 8 * 512 ** 3 < big < 1.25 * 2 * 8 * 512 ** 3
    assert 0.45 * big < f32 < 0.55 * big
    assert small < big
    batch = jg.jacobi_workspace_bytes_batch([(64, 64, 64), (48, 32, 16)],
                                            [("count", (2, 2, 2)), ("shape", (32, 32, 32))], "f32")
    assert batch > jg.jacobi_workspace_bytes((64, 64, 64), ("count", (2, 2, 2)), "f32")


def test_workspace_rejects_bad_split(lib):
    with pytest.raises(jg.JacobiError):
        jg.jacobi_workspace_bytes((10, 10, 10), ("count", (11, 1, 1)), "f64")
    with pytest.raises(jg.JacobiError):
        jg.jacobi_workspace_bytes((10, 10, 0), ("count", (1, 1, 1)), "f64")


def test_workspace_rejects_oversized_blocks(lib):
    # a block may span JACOBI_MAX_BLOCK_EXTENT = 32764 points per axis (its padded extent must fit the
    # 16-bit coordinates of a work item); 32765 pads to 32768 rows
    jg.jacobi_workspace_bytes((4, 32764, 1), ("count", (1, 1, 1)), "f32")
    for grid in [(4, 32765, 1), (32765, 4, 1), (4, 4, 32765)]:
        with pytest.raises(jg.JacobiError) as e:
            jg.jacobi_workspace_bytes(grid, ("count", (1, 1, 1)), "f32")
        assert e.value.code == jg.JACOBI_EINVAL
    # the same extent split in two is fine
    jg.jacobi_workspace_bytes((4, 65528, 1), ("count", (1, 2, 1)), "f32")


def test_autotune_path_rejects_bad_arguments(lib):
    # validated before any device work: a null handle, a path the search does
    # not cover, and a trial length below one iteration
    for args in ((None, "persistent", 8), (None, "explicit", 8), (None, "graph", 0)):
        with pytest.raises(jg.JacobiError):
            jg.jacobi_autotune_path(*args)
