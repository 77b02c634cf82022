"""The tuning text form (rng_parse_tune, and the BCN_RNG_TUNE override that
uses it) on the host: names and numbers, spacing, and every malformed input
rejected with a message, never half-applied.  No GPU."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def R():
    from paper_1206_1187_gb300 import _build
    _build.build()
    from paper_1206_1187_gb300 import rng
    return rng


def test_every_name_maps_to_its_enum(R):
    for key, table in (("step", R.STEP), ("conv", R.CONV), ("layout", R.LAYOUT),
                       ("skip", R.SKIP)):
        for name, code in table.items():
            if name == "auto":
                continue
            assert R.parse_tune(f"{key}={name}")[key] == code
            assert R.parse_tune(f"{key}={code}")[key] == code


def test_fields_spacing_and_defaults(R):
    t = R.parse_tune(" step=shared , conv=int,layout=tiled, skip=sqmul,depth=31,block=896,"
                     "grid=7,unit=64,chains=2,buffers=1 ")
    assert t == {"step": 3, "conv": 1, "layout": 1, "skip": 2, "depth": 31, "block": 896,
                 "grid": 7, "unit": 64, "chains": 2, "buffers": 1}
    assert R.parse_tune("") == {k: 0 for k in t}
    assert R.parse_tune("depth=4294967295")["depth"] == 2 ** 32 - 1
    assert R.parse_tune("depth=7,depth=9")["depth"] == 9  # the last one wins


@pytest.mark.parametrize("text,why", [
    ("foo=1", "unknown key"), ("step=fast", "bad value"), ("depth=-1", "bad value"),
    ("depth", "expected key=value"), ("depth=4294967296", "bad value"), ("step=", "bad value"),
    ("=3", "unknown key"), ("depth=1x", "bad value"), ("conv=INT", "bad value"),
])
def test_malformed_text_is_rejected(R, text, why):
    with pytest.raises(R.RNGError) as e:
        R.parse_tune(text)
    assert e.value.status == 1 and why in str(e.value)


def test_a_malformed_override_fails_every_call_loudly():
    """With BCN_RNG_TUNE set to text that does not parse, a call that takes
    defaults fails with RNG_EINVAL naming the variable (checked before any
    device is touched, so this runs without a GPU)."""
    code = ("from paper_1206_1187_gb300 import rng\n"
            "try:\n"
            "    rng.resolve_tune(1 << 20, 'f64')\n"
            "except rng.RNGError as e:\n"
            "    print(e.status, e)\n")
    env = dict(os.environ, BCN_RNG_TUNE="step=barrett,depth=fifteen")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("1 ") and "BCN_RNG_TUNE" in out.stdout
    assert "bad value 'fifteen' for depth" in out.stdout
