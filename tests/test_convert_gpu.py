"""The mixed form's integer-op format conversions equal IEEE round-to-nearest-
even (numpy's float32 cast) and exact widening, including ties, carries into
the exponent, the ends of the binary32 normal range, zeros and signs."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_08747_gb300 import build
    build.build()
    from paper_2410_08747_gb300 import mcx as m
    return m


def edge_cases():
    f32 = np.float32
    vals = [0.0, -0.0, 1.0, -1.0, 0.5, 1e-3, 123.456, float(np.finfo(f32).max),
            float(np.finfo(f32).tiny), 1e-40, 1e-45, 1e39, -1e39, 2.0**-126, 2.0**-127]
    rng = np.random.default_rng(3)
    base = rng.uniform(1, 2, 2000).astype(f32).astype(np.float64)
    ulp = np.spacing(base.astype(f32)).astype(np.float64)
    vals += list(base + 0.5 * ulp)                      # exact ties
    vals += list(base + 0.5 * ulp * (1 + 2.0**-20))     # just above ties
    vals += list(base + 0.5 * ulp * (1 - 2.0**-20))     # just below ties
    vals += list(np.nextafter(np.float64(2.0), 0.0) * 2.0 ** np.arange(-120, 120))  # carries
    vals += list(np.float64(np.finfo(f32).max) * (1 + np.array([1e-9, 2.0**-25, 2.0**-24])))
    e = rng.uniform(-140, 130, 20000)
    vals += list(rng.choice([-1.0, 1.0], 20000) * rng.uniform(1, 2, 20000) * 2.0 ** e)
    return np.array(vals, dtype=np.float64)


def test_round_and_widen_match_ieee(mcx):
    x = edge_cases()
    of, od = mcx.convert_fill(x)
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32)
    same = (of.view(np.uint32) == ref.view(np.uint32)) | (np.isnan(of) & np.isnan(ref))
    bad = np.nonzero(~same)[0]
    assert bad.size == 0, [(x[i], of[i], ref[i]) for i in bad[:5]]
    fin = np.isfinite(of)
    assert (od[fin] == of[fin].astype(np.float64)).all()
    assert (np.signbit(od) == np.signbit(of)).all()
