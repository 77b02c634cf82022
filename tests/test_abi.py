"""The C-ABI library loads and exports every entry point include/*.h declares;
host-side argument checks that need no GPU.  (No compute calls here.)"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        for m in re.finditer(r"\b([a-z_][a-z0-9_]*)\s*\(", text):
            name = m.group(1)
            # a declaration: the name follows a type, not a keyword or macro
            before = text[:m.start()].rstrip()
            if name.startswith("rng_") and (before.endswith("*") or re.search(r"[\w]$", before)):
                names.add(name)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1206_1187_gb300 import _build
    _build.build()
    from paper_1206_1187_gb300 import rng
    return rng


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("rng_create", "rng_generate", "rng_skip", "rng_destroy",
                     "rng_get_state", "rng_set_state", "rng_generate_at", "rng_sync",
                     "rng_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(lib.library_info.path)
    missing = [n for n in sorted(_declared_functions()) if not hasattr(raw, n)]
    assert not missing, missing


def test_seed_range_is_checked_on_the_host(lib):
    with pytest.raises(lib.RNGError) as e:
        lib.Stream(3 ** 33 + 99)
    assert e.value.status == 2
    with pytest.raises(lib.RNGError):
        lib.Stream(2 ** 53 + 1)
    s = lib.Stream(3 ** 33 + 100)
    assert s.state == (3 ** 33 + 100, 0)
    s2 = lib.Stream(2 ** 53)
    assert s2.state == (2 ** 53, 0)


def test_state_skip_and_checkpoint(lib):
    s = lib.Stream(3 ** 33 + 12345)
    s.skip(1000)
    s.skip(5)
    assert s.state == (3 ** 33 + 12345, 1005)
    s.set_state(8 * 10 ** 15, 77)
    assert s.state == (8 * 10 ** 15, 77)
    with pytest.raises(lib.RNGError) as e:
        s.set_state(5, 0)
    assert e.value.status == 2
    s.set_state(8 * 10 ** 15, 2 ** 64 - 10)
    with pytest.raises(lib.RNGError) as e:
        s.skip(11)
    assert e.value.status == 2
    assert s.state == (8 * 10 ** 15, 2 ** 64 - 10)


def test_empty_and_bad_pointer_calls_fail_before_any_launch(lib):
    raw = lib.lib
    s = lib.Stream(3 ** 33 + 100)
    # n = 0 is a no-op and touches no device
    assert raw.rng_generate(s._h, 0, 0, None) == 0
    assert s.state[1] == 0
    # NULL output, misaligned output, bad dtype, oversize n: all rejected
    assert raw.rng_generate(s._h, 10, 0, None) == 1
    assert raw.rng_generate(s._h, 10, 0, ctypes.c_void_p(4)) == 1
    assert raw.rng_generate(s._h, 10, 1, ctypes.c_void_p(2)) == 1
    assert raw.rng_generate(s._h, 10, 7, ctypes.c_void_p(4096)) == 1
    assert raw.rng_generate(s._h, (1 << 46) + 1, 0, ctypes.c_void_p(4096)) == 2
    assert s.state[1] == 0
    assert b"aligned" in raw.rng_last_error() or raw.rng_last_error()


def test_host_output_call_checks_arguments_first(lib):
    raw = lib.lib
    s = lib.Stream(3 ** 33 + 100)
    assert raw.rng_generate_to_host(s._h, 0, 0, None, 0, 0) == 0      # n = 0: no-op
    assert raw.rng_generate_to_host(s._h, 10, 0, None, 0, 0) == 1     # NULL output
    assert raw.rng_generate_to_host(s._h, 10, 0, ctypes.c_void_p(4), 0, 0) == 1  # misaligned
    buf = ctypes.create_string_buffer(128)
    addr = (ctypes.addressof(buf) + 15) // 16 * 16
    assert raw.rng_generate_to_host(s._h, 10, 0, ctypes.c_void_p(addr), 0, 9) == 1  # nbuf > 8
    assert raw.rng_generate_to_host(s._h, 10, 0, ctypes.c_void_p(addr), 2 ** 41, 2) == 1
    assert raw.rng_generate_to_host(s._h, 10, 7, ctypes.c_void_p(addr), 0, 2) == 1  # dtype
    assert s.state[1] == 0


def test_modulus_40_checks_arguments_first(lib):
    raw = lib.lib
    m40 = 3 ** 40
    vp = ctypes.c_void_p(4096)
    assert raw.rng40_generate_at(m40 + 99, 0, 10, 0, vp, None, None) == 2   # seed range
    assert raw.rng40_generate_at(m40 + 100, 0, 0, 0, None, None, None) == 0  # n = 0
    assert raw.rng40_generate_at(m40 + 100, 0, 10, 0, None, None, None) == 1
    assert raw.rng40_generate_at(m40 + 100, 0, 10, 0, ctypes.c_void_p(4), None, None) == 1
    assert raw.rng40_generate_at(m40 + 100, 0, 10, 5, vp, None, None) == 1  # dtype
    assert raw.rng40_generate_at(m40 + 100, 0, (1 << 46) + 1, 0, vp, None, None) == 2
    t = lib.make_tune(step="barrett")
    assert raw.rng40_generate_at(m40 + 100, 0, 10, 0, vp, None, ctypes.byref(t)) == 1
    assert b"3^40" in raw.rng_last_error()


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "bcn_rng.h"

#define CHECK(x) do { rng_status st_ = (x); if (st_ != RNG_OK) { \
    printf("FAIL %s: %d %s\n", #x, (int)st_, rng_last_error()); return 1; } } while (0)

int main(void) {
  bcn_stream *s = NULL;
  uint64_t a = 0, c = 0, off = 0, in_use = 0, live = 0;
  rng_tune t;
  bcn_pool *p = NULL;
  if (rng_create(5559060566555523ULL + 99, &s) != RNG_ERANGE) return 2;
  CHECK(rng_create(5559060566555523ULL + 100, &s));
  CHECK(rng_skip(s, 1000));
  CHECK(rng_get_state(s, &a, &c));
  if (a != 5559060566555523ULL + 100 || c != 1000) return 3;
  CHECK(rng_set_state(s, 1ULL << 53, 7));
  CHECK(rng_get_state(s, &a, &c));
  if (a != (1ULL << 53) || c != 7) return 4;
  CHECK(rng_destroy(s));
  CHECK(rng_parse_tune("step=barrett,depth=15", &t));
  if (t.step != RNG_STEP_BARRETT || t.depth != 15 || t.block != 0) return 5;
  if (rng_parse_tune("depth=x", &t) != RNG_EINVAL || strstr(rng_last_error(), "depth") == NULL)
    return 6;
  CHECK(rng_pool_create(1 << 20, 256, &p));
  CHECK(rng_pool_alloc(p, 1000, &off));
  CHECK(rng_pool_stats(p, &in_use, NULL, &live, NULL, NULL));
  if (off != 0 || in_use != 1024 || live != 1) return 7;
  CHECK(rng_pool_free(p, off));
  CHECK(rng_pool_destroy(p));
  printf("ok %d\n", rng_version());
  return 0;
}
"""


def test_device_api_checksum_checks_arguments_first(lib):
    """Seed range, output type, thread count and output pointer are checked on
    the host, before any launch (these calls need no GPU)."""
    import ctypes
    fn = lib.lib.rng_device_api_checksum
    buf = ctypes.cast((ctypes.c_uint64 * 128)(), ctypes.c_void_p)
    assert fn(3 ** 33 + 99, 0, 10, 0, buf, 128, None) == 2
    assert fn(2 ** 53 + 1, 0, 10, 0, buf, 128, None) == 2
    for threads in (0, 100, 129):
        assert fn(3 ** 33 + 100, 0, 10, 0, buf, threads, None) == 1
    for dt in (2, 3, -1):
        assert fn(3 ** 33 + 100, 0, 10, dt, buf, 128, None) == 1
    assert fn(3 ** 33 + 100, 0, 10, 0, None, 128, None) == 1
    runs = lib.lib.rng_device_api_f32_runs
    out = ctypes.cast((ctypes.c_float * 64)(), ctypes.c_void_p)
    assert runs(3 ** 33 + 99, 0, 10, out, 128, None) == 2
    assert runs(3 ** 33 + 100, 0, 10, out, 96, None) == 1
    assert runs(3 ** 33 + 100, 0, 10, None, 128, None) == 1
    assert runs(3 ** 33 + 100, 0, 0, None, 128, None) == 0  # n = 0: nothing to write


def test_the_boundary_is_usable_from_plain_c(lib, tmp_path):
    """The header compiles as C99 with warnings as errors, and a C program
    linked against the library drives its host-side entry points."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib.library_info.path)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                        "-L", libdir, "-lbcn_rng", f"-Wl,-rpath,{libdir}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip() == f"ok {lib.version()}"


DEVICE_KERNEL = r"""
#include "bcn_device.cuh"

__global__ void user_sim(unsigned long long seed, unsigned long long first, double* f64,
                         float* f32, unsigned long long* st, float* runs) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  bcn_device::Stream g = bcn_device::make_stream(seed, first, 4ull * t);
  bcn_device::Stream h = g, k = g;
  for (int i = 0; i < 4; ++i) {
    f64[4 * t + i] = bcn_device::next_f64(g);
    f32[4 * t + i] = bcn_device::next_f32(h);
    st[4 * t + i] = bcn_device::next_state(k);
  }
  float w[8];
  bcn_device::f32_run<8>(seed, first, 8ull * t, w);
  for (int i = 0; i < 8; ++i) runs[8 * t + i] = w[i];
}
"""


def test_device_header_is_usable_from_a_user_kernel(tmp_path):
    """include/bcn_device.cuh compiles for sm_103a in a user's kernel with only
    include/ on the include path (no GPU needed to compile)."""
    import subprocess
    from paper_1206_1187_gb300 import _build
    try:
        nvcc = _build._nvcc()
    except RuntimeError:
        pytest.skip("no nvcc")
    src = tmp_path / "user.cu"
    src.write_text(DEVICE_KERNEL)
    r = subprocess.run([nvcc] + _build.ARCH + ["-std=c++17", "-O3", "-I",
                                               os.path.join(ROOT, "include"), "-c", str(src),
                                               "-o", str(tmp_path / "user.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
