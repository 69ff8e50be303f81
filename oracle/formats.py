"""Decoders for the storage formats of the samples V, written from the formats' bit-level
definitions. The paper works in FP64 throughout; these formats belong to the reduced-precision
storage of V (BF16, FP8 e4m3 with one FP32 scale per sample), and the oracle evaluates Alg. 2 on
the decoded values exactly, in FP64.

Test infrastructure only (see the package docstring).
"""

import numpy as np


def decode_bf16(bits):
    """bfloat16 bit patterns (uint16) -> FP64. A bfloat16 is the upper 16 bits of an IEEE
    binary32, so widening is exact."""
    b = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << np.uint32(16)
    return b.view(np.float32).astype(np.float64)


def decode_e4m3(bits):
    """OCP 8-bit floating point, E4M3 variant (1 sign, 4 exponent bits with bias 7, 3 mantissa
    bits; no infinities; S.1111.111 is NaN) -> FP64.

    normal   (e > 0): (-1)^s * (1 + m/8) * 2^(e - 7)
    subnormal(e = 0): (-1)^s * (m/8) * 2^(1 - 7)
    """
    b = np.asarray(bits, dtype=np.uint8).astype(np.int64)
    s = (b >> 7) & 1
    e = (b >> 3) & 0xF
    m = b & 0x7
    mag = np.where(e > 0, (1.0 + m / 8.0) * np.exp2(e - 7.0), (m / 8.0) * np.exp2(-6.0))
    mag = np.where((e == 0xF) & (m == 0x7), np.nan, mag)
    return np.where(s == 1, -mag, mag)


def dequantize_e4m3(q_bits, scale):
    """v_l = s_l * q_l for sample-major codes q (p x n, uint8) and per-sample scales s (p).
    Returns the p x n FP64 samples."""
    q = decode_e4m3(q_bits)
    return q * np.asarray(scale, dtype=np.float64)[:, None]
