"""CPU checks of the benchmark's CPU throughput baseline (not a parity test of the
CUDA path): the batched FP32 NumPy L-MMSE of ``bench.numpy32_equalize`` computes
what the oracle computes (unbiased PD and FD with optimal fusion) to FP32
accuracy, so its symbols/s line times the same work."""
import numpy as np

import bench
from oracle import lmmse
from paper_1808_04473_gb300 import synth


def test_numpy_fp32_baseline_matches_the_oracle():
    p = synth.make_problem(64, 8, 4, 30, 5, snr_db=12.0, bits=4, seed=41)
    for fd, f in ((False, lmmse.equalize_pd), (True, lmmse.equalize_fd)):
        z, s2 = bench.numpy32_equalize(p.H, p.y, p.N0, p.Es, p.C, fd)
        o = f(p.H, p.y, p.N0, p.Es, p.C, "unbiased")
        ez = np.linalg.norm((z - o["z"]).reshape(30, -1), axis=1) / np.linalg.norm(o["z"].reshape(30, -1), axis=1)
        es = np.abs(s2 - o["sigma2"]).max() / np.abs(o["sigma2"]).max()
        assert ez.max() < 1e-5 and es < 1e-5, (fd, ez.max(), es)


def test_error_measures():
    o = np.ones((2, 4), np.complex128)
    g = o.copy()
    g[1, 2] += 1e-3
    nrm, ent = bench._errors(g, o)
    assert abs(ent - 1e-3) < 1e-12 and abs(nrm - 1e-3 / 2) < 1e-12


def test_lama_flop_count():
    # Per received vector and cluster, U = 16, 16-QAM (two bits per PAM axis),
    # T = 8: eight products of 8 U^2 = 2048 flops and seven denoiser steps of
    # U (2 * 4 * 6 + 10) = 928 flops: 16 384 + 6 496.
    import bench
    assert bench.lama_flops(16, 4, 8) == 16384 + 6496 == 22880
    # T = 1: one product, no denoiser step.
    assert bench.lama_flops(8, 2, 1) == 8 * 64
