"""The C-ABI library builds, loads and exports what include/*.h declares (CPU only)."""
import ast
import ctypes
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1803_09835_gb300")


@pytest.fixture(scope="module")
def lib():
    from paper_1803_09835_gb300 import _build, _lib
    _build.build()
    return ctypes.CDLL(_lib.LIB_PATH)


def test_every_declared_symbol_is_exported(lib):
    from paper_1803_09835_gb300 import _lib
    names = _lib.header_functions()
    assert "fast_detect" in names and "fast_search" in names and len(names) >= 14
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/*.h but not exported"


def test_binding_covers_the_header():
    from paper_1803_09835_gb300 import _lib
    for n in _lib.header_functions():
        assert hasattr(_lib, n), f"no Python binding named {n}"


def test_product_never_touches_the_oracle():
    # The product path may not import, load or run anything under oracle/.
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            path = os.path.join(dirpath, f)
            if f.endswith(".py"):
                tree = ast.parse(open(path).read())
                for node in ast.walk(tree):
                    if isinstance(node, ast.Import):
                        assert not any(a.name.split(".")[0] == "oracle" for a in node.names), path
                    if isinstance(node, ast.ImportFrom):
                        assert (node.module or "").split(".")[0] != "oracle", path
            if f.endswith((".cu", ".cuh", ".h", ".py")):
                assert "liboracle" not in open(path).read(), path


def test_no_gpu_means_an_error_not_a_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1803_09835_gb300 import FastError, Searcher
    with pytest.raises(FastError):
        Searcher(dict(D=2048, K=100, b=16, r=4, kind=0, seed=1, v=2, excl=5, occ_num=0, occ_den=1))


def test_closing_a_searcher_frees_what_it_made():
    # a result may not outlive its context: the wrapper frees every live
    # object of a context before destroying it (checked without a GPU on a
    # stand-in object)
    import paper_1803_09835_gb300 as pkg

    class Obj:
        freed = 0

        def free(self):
            Obj.freed += 1

    s = pkg.Searcher.__new__(pkg.Searcher)
    import weakref
    s._live = weakref.WeakSet()
    keep = [Obj(), Obj()]
    for o in keep:
        pkg._track(s, o)
    s.ctx = None  # no context: close() has nothing to destroy
    s.close()
    assert Obj.freed == 0  # without a context nothing is touched
    calls = []
    pkg_destroy = pkg.fast_destroy
    try:
        pkg.fast_destroy = lambda ctx: calls.append(ctx)
        s.ctx = "ctx"
        s.close()
    finally:
        pkg.fast_destroy = pkg_destroy
    assert Obj.freed == 2 and calls == ["ctx"] and s.ctx is None
