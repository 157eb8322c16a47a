"""The table-driven FP64 logarithm the Neo-Hookean kernels take ln det F with.

CPU: the committed table matches its definition (interval centres, reciprocals
rounded to double, -ln of the rounded reciprocal, the ln 2 shift above sqrt 2).
GPU: the device function against the host libm logarithm and the hardware
library's, in units in the last place, over the argument ranges that matter
(det F near 1 from both sides, interval edges, sqrt 2, powers of two, the whole
normal and subnormal range)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_1604_05872_gb300", "csrc", "log_table.h")


def read_table():
    src = open(HEADER).read()
    split = int(re.search(r"kLogSplit = (\d+)", src).group(1))
    hi = float.fromhex(re.search(r"kLn2Hi = ([0-9a-fx.p+-]+);", src).group(1))
    lo = float.fromhex(re.search(r"kLn2Lo = ([0-9a-fx.p+-]+);", src).group(1))
    rows = [(float.fromhex(a), float.fromhex(b)) for a, b in re.findall(r"\{(-?0x[0-9a-fx.p+-]+), (-?0x[0-9a-fx.p+-]+)\}", src)]
    return split, hi, lo, rows


def test_table_matches_its_definition():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    split, hi, lo, rows = read_table()
    assert len(rows) == 128 and 1 + split / 128 <= 2 ** 0.5 < 1 + (split + 1) / 128  # split at the sqrt 2 interval
    ln2 = mpmath.log(2)
    assert abs(mpmath.mpf(hi) + mpmath.mpf(lo) - ln2) < mpmath.mpf(2) ** -95
    assert float(mpmath.mpf(hi) * 2 ** 42) == round(float(mpmath.mpf(hi) * 2 ** 42))  # k * hi exact for |k| < 2^11
    for j, (inv, L) in enumerate(rows):
        c = 1 if j == 0 else 2 if j == 127 else 1 + (2 * j + 1) / 256
        assert inv == float(1 / mpmath.mpf(c))
        want = -mpmath.log(mpmath.mpf(inv)) - (ln2 if j >= split else 0)
        assert L == float(want), j
        # every mantissa of the interval is within 2^-7 of its centre, relative
        lo_m, hi_m = 1 + j / 128, 1 + (j + 1) / 128
        assert max(abs(lo_m * inv - 1), abs(hi_m * inv - 1)) <= 2 ** -7


def ulp_error(got, want):
    """|got - want| in units of the last place of want (float64)."""
    return np.abs(got - want) / np.spacing(np.abs(want))


def arguments():
    rng = np.random.default_rng(160405872)
    parts = [
        1 + rng.uniform(-0.3, 0.3, 200000),                          # det F of the workloads
        1 + rng.uniform(-1e-6, 1e-6, 50000),                         # nearly volume-preserving
        np.nextafter(1.0, 2.0) + np.arange(1000) * np.spacing(1.0),  # just above 1
        np.nextafter(1.0, 0.0) - np.arange(1000) * np.spacing(0.5),  # just below 1
        np.exp(rng.uniform(-700, 700, 100000)),                      # whole normal range
        np.ldexp(1.0, np.arange(-1074, 1024)).astype(np.float64),    # powers of two (subnormals too)
        rng.uniform(0, 1, 20000) * np.ldexp(1.0, -1022),             # subnormals
        np.array([np.sqrt(2.0), np.nextafter(np.sqrt(2.0), 0), np.nextafter(np.sqrt(2.0), 3), 0.5 * np.sqrt(2.0)]),
    ]
    # both edges of every table interval, in [1, 2) and scaled by 1/2 (k = -1)
    edges = 1 + np.arange(129) / 128
    parts += [edges, np.nextafter(edges, 0), np.nextafter(edges, 3), 0.5 * edges, 0.5 * np.nextafter(edges, 0)]
    x = np.concatenate(parts)
    return x[(x > 0) & np.isfinite(x)]


@pytest.mark.gpu
def test_device_log_against_host_and_hardware_library(fea):
    import torch
    x = arguments()
    xt = torch.from_numpy(x).cuda()
    got = fea.log_f64(xt).cpu().numpy()
    fea.sync()
    host = np.log(x)
    lib = torch.log(xt).cpu().numpy()
    nz = host != 0
    assert np.all(got[~nz] == 0.0)  # ln 1 = 0 exactly
    e_host = ulp_error(got[nz], host[nz])
    e_lib = ulp_error(got[nz], lib[nz])
    assert e_host.max() <= 2.0, (x[nz][e_host.argmax()], e_host.max())
    assert e_lib.max() <= 3.0, (x[nz][e_lib.argmax()], e_lib.max())
    # near 1 the result keeps its relative accuracy (no cancellation with the table term)
    near = (np.abs(x - 1) < 1e-3) & nz
    assert np.max(np.abs(got[near] - host[near]) / np.abs(host[near])) <= 4.5e-16
