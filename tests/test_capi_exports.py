"""The C-ABI library builds for sm_103a and exports every function include/enuf.h
declares (CPU only: loads the library, makes no compute call)."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "enuf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:enuf_status|void|int|const char\*)\s+\**\s*((?:enuf|dpd)_\w+)\s*\(", src, re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_1303_4523_gb300 import build
    lib_path = build.build()
    declared = _declared()
    assert len(declared) >= 20
    lib = ctypes.CDLL(lib_path)
    for name in declared:
        assert hasattr(lib, name), name
    nm = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T ((?:enuf|dpd)_\w+)", nm))
    assert set(declared) == exported


def test_binding_names_match_header():
    from paper_1303_4523_gb300 import build
    build.build()
    from paper_1303_4523_gb300 import enuf
    assert sorted(enuf.EXPORTED) == _declared()


def test_status_strings_and_invalid_params_without_gpu():
    """Parameter validation and footprints are host logic: no GPU needed."""
    from paper_1303_4523_gb300 import build
    build.build()
    from paper_1303_4523_gb300 import enuf
    assert enuf.lib.enuf_status_string(1) == b"invalid argument"
    ok = enuf.make_params(L=30.0, alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, M=48, p=4)
    b = enuf.enuf_footprint(ok, 81000)
    assert 10e6 < b < 400e6
    b32 = enuf.enuf_footprint(enuf.make_params(L=30.0, alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, M=48, p=4,
                                               prec="fp32"), 81000)
    assert b32 < b
    for bad in (dict(L=-1.0), dict(r_cut=16.0), dict(M=47), dict(p=0), dict(p=9), dict(sigma_s=3),
                dict(alpha=0.0), dict(kmask=2)):
        kw = dict(L=30.0, alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, M=48, p=4)
        kw.update(bad)
        try:
            enuf.enuf_footprint(enuf.make_params(**kw), 100)
        except enuf.EnufError as e:
            assert e.status == 1, bad
        else:
            raise AssertionError(f"accepted {bad}")
    # bead capacity: per-bead components are indexed as int, so n_max <= 2^29
    assert enuf.enuf_footprint(ok, 1 << 29) > 16 * (1 << 29)
    for bad_n in (-1, (1 << 29) + 1):
        try:
            enuf.enuf_footprint(ok, bad_n)
        except enuf.EnufError as e:
            assert e.status == 1, bad_n
        else:
            raise AssertionError(f"accepted n_max = {bad_n}")
    # the allocation-failure injection is host state: set and cleared without a GPU
    enuf.debug_fail_allocs(2, after=1)
    enuf.debug_fail_allocs(0)
    for bad_args in ((-1, 0), (0, -1)):
        try:
            enuf.debug_fail_allocs(*bad_args)
        except enuf.EnufError as e:
            assert e.status == 1
        else:
            raise AssertionError(f"accepted {bad_args}")
    # a grid with a prime factor other than 2, 3, 5 is unsupported
    try:
        enuf.enuf_footprint(enuf.make_params(L=30.0, alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, M=14, p=4), 10)
    except enuf.EnufError as e:
        assert e.status == 5
    else:
        raise AssertionError("accepted n = 28")


def test_method_switches_are_validated_without_gpu():
    """The method switches and the tile edge are checked by the plan's host
    logic; gradient mode holds one force field instead of three."""
    from paper_1303_4523_gb300 import build
    build.build()
    from paper_1303_4523_gb300 import enuf
    base = dict(L=30.0, alpha=0.975, r_cut=3.0, beta=4.0, kappa=1.1, M=48, p=4)
    for bad in (dict(deriv=2), dict(slater_k=1, beta=0.0), dict(slater_k=2), dict(fft_path=2), dict(fft_radix=3), dict(tile=7),
                dict(tile=48), dict(tile=3)):
        kw = dict(base)
        kw.update(bad)
        try:
            enuf.enuf_footprint(enuf.make_params(**kw), 100)
        except enuf.EnufError as e:
            assert e.status == 1, bad
        else:
            raise AssertionError(f"accepted {bad}")
    for ok in (dict(deriv=1), dict(slater_k=1), dict(fft_path=1), dict(fft_radix=1), dict(fft_radix=2), dict(tile=12), dict(tile=24)):
        kw = dict(base)
        kw.update(ok)
        assert enuf.enuf_footprint(enuf.make_params(**kw), 100) > 0, ok
    n3 = 96 ** 3
    for prec, esz in (("fp64", 8), ("fp32", 4)):
        ik = enuf.enuf_footprint(enuf.make_params(prec=prec, **base), 81000)
        grad = enuf.enuf_footprint(enuf.make_params(prec=prec, deriv=1, **base), 81000)
        assert ik - grad >= 2 * n3 * esz   # two real fields fewer (and their spectra)


def test_checked_build_exports_the_same_api():
    """The debug build (-DENUF_CHECK, device index checks) compiles and exports
    the same functions; each build reports whether it carries the checks."""
    from paper_1303_4523_gb300 import build
    rel = ctypes.CDLL(build.build())
    chk = ctypes.CDLL(build.build(check=True))
    for name in _declared():
        assert hasattr(chk, name), name
    assert rel.enuf_built_with_checks() == 0 and chk.enuf_built_with_checks() == 1
