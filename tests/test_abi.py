"""Host-side checks of the C ABI: the library loads, exports every declared symbol, and
rejects invalid arguments before touching the GPU (no device needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "htlr.h")).read()
    pat = r"^(?:const\s+char\s*\*|long\s+long|int|void|double)\s*\*?\s*(htlr_[a-z_]+)\s*\("
    return sorted(set(re.findall(pat, src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    from paper_2508_05958_gb300 import htlr
    L = htlr.load()
    names = declared_symbols()
    assert set(names) == set(htlr.SYMBOLS), names
    for name in names:
        assert hasattr(L, name), name


def test_header_compiles_as_c():
    import subprocess
    import tempfile
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "t.c")
        open(c, "w").write('#include "htlr.h"\nint main(void){htlr_stats s; (void)s; '
                           'return HTLR_OK;}\n')
        r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I",
                            os.path.join(ROOT, "include"), "-c", c, "-o",
                            os.path.join(td, "t.o")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


@pytest.mark.parametrize("kw,code", [
    (dict(d=4), -1), (dict(d=1), -1), (dict(n=30), -1), (dict(n=24, leaf=8), -1),
    (dict(n=8, leaf=8), -1), (dict(r=0), -1), (dict(r=17), -1), (dict(ktype=9), -1),
    (dict(ktype=3, kparam=0.0), -1), (dict(ktype=4, kparam=2.5), -1),
    (dict(eta=float("nan")), -1), (dict(quad_order=65), -1), (dict(orth=3), -1),
])
def test_construct_rejects_invalid_arguments(kw, code):
    from paper_2508_05958_gb300 import htlr
    args = dict(ktype=1, d=3, n=32, leaf=4, r=5, eta=1.0)
    extra = {}
    for k in ("kparam", "quad_order", "orth"):
        if k in kw:
            extra[k] = kw.pop(k)
    args.update(kw)
    with pytest.raises(htlr.HTLRError) as ei:
        htlr.htlr_construct(args["ktype"], args["d"], args["n"], args["leaf"], args["r"],
                            args["eta"], **extra)
    assert ei.value.code == code
    assert htlr.htlr_last_error()


def test_null_and_dead_handles():
    from paper_2508_05958_gb300 import htlr
    L = htlr.load()
    L.htlr_free(None)                                   # no-op
    assert L.htlr_matvec(None, None, None, 1) == htlr.HTLR_EINVAL
    bogus = ctypes.c_void_p(0x1234)
    assert L.htlr_matvec(bogus, None, None, 1) == htlr.HTLR_EINVAL
    L.htlr_free(bogus)                                  # not live: ignored, reported
    assert "not a live" in htlr.htlr_last_error()
    s = htlr.htlr_stats()
    assert L.htlr_info(bogus, ctypes.byref(s)) == htlr.HTLR_EINVAL
    assert L.htlr_last_launch_count(bogus) == -1
    k = htlr.htlr_kernel(1, 1.0, 0.0)
    assert L.htlr_construct(None, ctypes.byref(k), 3, 32, None, 4, 5, 1.0) == htlr.HTLR_EINVAL


def test_product_and_oracle_share_no_code():
    """The library and its binding never reach the CPU oracle, and the oracle includes
    nothing of the library: the two are independent implementations."""
    import glob
    pkg = os.path.join(ROOT, "paper_2508_05958_gb300")
    files = [p for ext in ("py", "cu", "cuh", "h") for p in
             glob.glob(os.path.join(pkg, "**", "*." + ext), recursive=True)]
    files += [os.path.join(ROOT, "include", "htlr.h")]
    assert len(files) > 10
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b|from\s+\.\.\s*import\s+oracle)|"
                     r"htlr_oracle|liboracle", re.M)
    for p in files:
        assert not pat.search(open(p).read()), p
    src = open(os.path.join(ROOT, "oracle", "htlr_oracle.c")).read()
    includes = re.findall(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', src, flags=re.M)
    assert includes and all(not i.startswith("htlr") and "/" not in i for i in includes), includes


def test_loading_the_library_does_not_import_the_oracle():
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r); import paper_2508_05958_gb300 as p; p.load(); "
            "print('oracle' in sys.modules)" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd="/")
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "False"
