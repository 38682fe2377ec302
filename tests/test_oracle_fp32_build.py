"""The FP32 build of the oracle source (liboracle32.so) is the plain FP32
CPU program the benchmark times beside the FP64 oracle.  It is not a
reference, so it is only checked to run the same algorithm: on a
well-conditioned frame its estimates agree with the FP64 build to FP32
accuracy, and the FP64 build is unchanged by the type switch (its pins are
in test_oracle_pins.py)."""
import numpy as np

import oracle
import synth


def test_fp32_build_agrees_with_fp64_build():
    f = synth.uplink_frame(16, 6, 128, 8, 16, 15.0, seed=31)
    H = f["H"].astype(np.complex64)
    y = f["y"].astype(np.complex64)
    ref = oracle.admm_ul(H.astype(np.complex128), y.astype(np.complex128), C=8, rho=1.0, N0=f["N0"], T_max=3)
    x32 = oracle.admm_ul_fp32(H, y, C=8, rho=1.0, N0=f["N0"], T_max=3)
    assert x32.dtype == np.complex64
    rel = np.linalg.norm(x32.astype(np.complex128) - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
    assert rel.max() < 1e-4
    assert rel.max() > 0.0          # it really ran in FP32


def test_fp32_build_rejects_bad_arguments():
    H = np.zeros((2, 16, 4), np.complex64)
    y = np.zeros((2, 3, 16), np.complex64)
    try:
        oracle.admm_ul_fp32(H, y, C=3, rho=1.0, N0=0.1)       # B not a multiple of C
    except ValueError as e:
        assert "bad argument" in str(e)
    else:
        raise AssertionError("expected a ValueError")
