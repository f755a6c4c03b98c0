"""The exact int16 -> float decode that the first FFT pass uses for odd samples of binary-phase
codes, checked on the host for every int16 value and both chip signs: XOR 0x8000 makes the
sample the offset-binary u = v + 2^15; its 16 bits in the low mantissa of 1.5 * 2^23 (float bits
0x4B40_0000, the chip's sign in bit 31) give +-(1.5 * 2^23 + u) exactly, and adding
-(1.5 * 2^23 + 2^15) (float bits 0xCB40_8000, sign flipped with the chip's) leaves +-v.  The
constants are the ones in the kernel's decode; the GPU parity tests run the kernel itself."""
import numpy as np

CS = 0x4B400000      # 1.5 * 2^23
KS = 0xCB408000      # -(1.5 * 2^23 + 2^15)


def _decode(words: np.ndarray, sbit: int) -> tuple:
    """Both components of the packed (I low, Q high) int16 pairs, as the kernel forms them."""
    wb = words ^ np.uint32(0x80008000)
    cs = np.uint32(CS ^ sbit)
    ks = np.array([KS ^ sbit], dtype=np.uint32).view(np.float32)[0]
    fi = ((wb & np.uint32(0xFFFF)) | (cs & np.uint32(0xFFFF0000))).view(np.float32)   # bytes wb.0, wb.1, cs.2, cs.3
    fq = ((wb >> np.uint32(16)) | (cs & np.uint32(0xFFFF0000))).view(np.float32)      # bytes wb.2, wb.3, cs.2, cs.3
    return (fi + ks).astype(np.float64), (fq + ks).astype(np.float64)


def test_decode_is_exact_for_every_int16_and_both_signs():
    v = np.arange(-32768, 32768, dtype=np.int64)
    q = v[::-1].copy()                          # pair every I with a different Q
    words = ((v & 0xFFFF) | ((q & 0xFFFF) << 16)).astype(np.uint32)
    for sbit, s in ((0, 1), (0x80000000, -1)):
        i_dec, q_dec = _decode(words, sbit)
        assert np.array_equal(i_dec, s * v.astype(np.float64))
        assert np.array_equal(q_dec, s * q.astype(np.float64))


def test_magic_constants():
    as_float = lambda bits: float(np.array([bits], dtype=np.uint32).view(np.float32)[0])
    assert as_float(CS) == 1.5 * 2**23
    assert as_float(KS) == -(1.5 * 2**23 + 2**15)
    # the sum's operands stay integers below 2^24: every partial result is exact in FP32
    assert 1.5 * 2**23 + 2**16 < 2**24
