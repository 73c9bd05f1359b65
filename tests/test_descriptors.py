"""CPU checks of the tensor-core encodings the kernels hand to tcgen05.

A host-only program (nvcc, no GPU) prints the instruction descriptors of the
FP8 (kind::f8f6f4) and FP4 (kind::mxf4, block-scaled) MMAs, the 128-byte
swizzled shared-memory matrix descriptor, the operand codes of +1 and -1,
the bit-spreading helpers that assemble the sign codes of 4 or 8 spins and
the band-order tile map of the one-step kernels.
The test decodes each field with the bit layout of the PTX ISA's tcgen05
descriptor tables, written out here independently of the library's helpers,
and the operand codes with the OCP MX element formats (e4m3, e2m1, UE8M0).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2203_08361_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

PROGRAM = r"""
#include <stdio.h>
#include "hsb_ptx.cuh"
#include "hsb_device.cuh"
#include "hsb_sched.cuh"
int main()
{
    printf("mxf4_128_192 %u\n", hsb::ptx::idesc_mxf4_e2m1(128, 192));
    printf("mxf4_128_256 %u\n", hsb::ptx::idesc_mxf4_e2m1(128, 256));
    printf("mxf4_256_192 %u\n", hsb::ptx::idesc_mxf4_e2m1(256, 192));
    printf("e4m3_256_256 %u\n", hsb::ptx::idesc_e4m3_f32(256, 256));
    printf("e4m3_128_256 %u\n", hsb::ptx::idesc_e4m3_f32(128, 256));
    printf("e4m3_256_128 %u\n", hsb::ptx::idesc_e4m3_f32(256, 128));
    printf("sw128_at_9216 %llu\n", (unsigned long long)hsb::ptx::sw128_desc(9216u));
    printf("fp4_plus %u\n", (unsigned)hsb::kFp4PlusOne);
    printf("fp4_minus %u\n", (unsigned)hsb::kFp4MinusOne);
    printf("fp8_plus %u\n", (unsigned)hsb::kFp8PlusOne);
    printf("fp8_minus %u\n", (unsigned)hsb::kFp8MinusOne);
    // the band-order tile map of the one-step kernels over (nmb, nrb, band):
    // every tile once; prints the count of shapes where it is not a bijection
    int bad_maps = 0, shapes = 0;
    for (int nmb = 1; nmb <= 70; nmb += 3)
        for (int nrb = 1; nrb <= 40; ++nrb)
            for (int band = 1; band <= nrb; band += (band < 8 ? 1 : 5)) {
                static unsigned char seen[70 * 40];
                const int ntiles = nmb * nrb;
                for (int i = 0; i < ntiles; ++i)
                    seen[i] = 0;
                bool ok = true;
                for (int t = 0; t < ntiles; ++t) {
                    int mb = -1, rb = -1;
                    hsb::tile_coords(t, nmb, nrb, band, mb, rb);
                    if (mb < 0 || mb >= nmb || rb < 0 || rb >= nrb || seen[mb * nrb + rb]++)
                        ok = false;
                }
                bad_maps += !ok;
                ++shapes;
            }
    printf("tile_map_shapes %d\n", shapes);
    printf("tile_map_bad %d\n", bad_maps);
    // one shape in full: nmb = 3, nrb = 5, band = 2 (bands of 2, 2, 1 blocks)
    for (int t = 0; t < 15; ++t) {
        int mb, rb;
        hsb::tile_coords(t, 3, 5, 2, mb, rb);
        printf("tile_3_5_2_%d %d\n", t, mb * 5 + rb);
    }
    for (unsigned b = 0; b < 256; ++b) {
        printf("spread4_%u %u\n", b, hsb::spread4_bytes(b));
        printf("spread8_%u %u\n", b, hsb::spread8_nibbles(b));
        printf("bmask4_%u %u\n", b, hsb::byte_mask4(b));
        printf("nmask8_%u %u\n", b, hsb::nibble_mask8(b));
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def values(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("desc")
    src, exe = d / "desc.cu", d / "desc"
    src.write_text(PROGRAM)
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", CSRC, "-I", INCLUDE, str(src), "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


def bits(v, lo, hi):
    """Field of bits lo..hi (inclusive)."""
    return (v >> lo) & ((1 << (hi - lo + 1)) - 1)


def decode_block_scaled_idesc(v):
    # tcgen05 instruction descriptor for .kind::mxf8f6f4 / mxf4 / mxf4nvf4
    return {
        "reserved_0_1": bits(v, 0, 1), "sparse": bits(v, 2, 2), "reserved_3": bits(v, 3, 3),
        "b_scale_id": bits(v, 4, 5), "reserved_6": bits(v, 6, 6),
        "a_fmt": bits(v, 7, 9), "b_fmt": bits(v, 10, 12),
        "neg_a": bits(v, 13, 13), "neg_b": bits(v, 14, 14),
        "a_mn_major": bits(v, 15, 15), "b_mn_major": bits(v, 16, 16),
        "n_shr3": bits(v, 17, 22), "scale_ue8m0": bits(v, 23, 23),
        "m_shr4": bits(v, 24, 28), "a_scale_id": bits(v, 29, 30), "k_dim": bits(v, 31, 31),
    }


def decode_f8f6f4_idesc(v):
    # tcgen05 instruction descriptor for .kind::f16 / tf32 / f8f6f4 / i8
    return {
        "sparse_sel": bits(v, 0, 1), "sparse": bits(v, 2, 2), "saturate": bits(v, 3, 3),
        "d_fmt": bits(v, 4, 5), "reserved_6": bits(v, 6, 6),
        "a_fmt": bits(v, 7, 9), "b_fmt": bits(v, 10, 12),
        "neg_a": bits(v, 13, 13), "neg_b": bits(v, 14, 14),
        "a_mn_major": bits(v, 15, 15), "b_mn_major": bits(v, 16, 16),
        "n_shr3": bits(v, 17, 22), "reserved_23": bits(v, 23, 23),
        "m_shr4": bits(v, 24, 28), "reserved_29": bits(v, 29, 29), "max_shift": bits(v, 30, 31),
    }


E2M1 = 1  # element format code of e2m1 in the block-scaled descriptor
E4M3 = 0  # element format code of e4m3 in the f8f6f4 descriptor
F32 = 1   # accumulator format code of f32


@pytest.mark.parametrize("key,M,N", [("mxf4_128_192", 128, 192), ("mxf4_128_256", 128, 256),
                                     ("mxf4_256_192", 256, 192)])
def test_mxf4_instruction_descriptor_fields(values, key, M, N):
    f = decode_block_scaled_idesc(values[key])
    assert f == {
        "reserved_0_1": 0, "sparse": 0, "reserved_3": 0, "b_scale_id": 0, "reserved_6": 0,
        "a_fmt": E2M1, "b_fmt": E2M1, "neg_a": 0, "neg_b": 0,
        "a_mn_major": 0, "b_mn_major": 0,          # K-major A and B
        "n_shr3": N // 8, "scale_ue8m0": 1,        # UE8M0 block scales
        "m_shr4": M // 16, "a_scale_id": 0, "k_dim": 0,
    }


@pytest.mark.parametrize("key,M,N", [("e4m3_128_256", 128, 256), ("e4m3_256_128", 256, 128),
                                     ("e4m3_256_256", 256, 256)])
def test_f8f6f4_instruction_descriptor_fields(values, key, M, N):
    f = decode_f8f6f4_idesc(values[key])
    assert f == {
        "sparse_sel": 0, "sparse": 0, "saturate": 0, "d_fmt": F32, "reserved_6": 0,
        "a_fmt": E4M3, "b_fmt": E4M3, "neg_a": 0, "neg_b": 0, "a_mn_major": 0,
        "b_mn_major": 0, "n_shr3": N // 8, "reserved_23": 0, "m_shr4": M // 16,
        "reserved_29": 0, "max_shift": 0,
    }


def test_shared_memory_descriptor_fields(values):
    # matrix descriptor: start >> 4 (0-13), leading byte offset >> 4 (16-29),
    # stride byte offset >> 4 (32-45), fixed 0b01 (46-47), base offset
    # (49-51), leading-offset mode (52), swizzle (61-63; 2 = 128-byte)
    v = values["sw128_at_9216"]
    assert bits(v, 0, 13) << 4 == 9216
    assert bits(v, 16, 29) == 1
    assert bits(v, 32, 45) << 4 == 1024      # 8 rows of 128 bytes
    assert bits(v, 46, 47) == 1
    assert bits(v, 49, 51) == 0 and bits(v, 52, 52) == 0
    assert bits(v, 61, 63) == 2
    assert bits(v, 14, 15) == 0 and bits(v, 30, 31) == 0 and bits(v, 53, 60) == 0


def decode_e2m1(code):
    """OCP MX e2m1: sign, 2 exponent bits (bias 1), 1 mantissa bit."""
    s, e, m = (code >> 3) & 1, (code >> 1) & 3, code & 1
    mag = 0.5 * m if e == 0 else 2.0 ** (e - 1) * (1 + m / 2)
    return -mag if s else mag


def decode_e4m3(code):
    """OCP e4m3 (finite values): sign, 4 exponent bits (bias 7), 3 mantissa bits."""
    s, e, m = (code >> 7) & 1, (code >> 3) & 15, code & 7
    mag = 2.0 ** -6 * (m / 8) if e == 0 else 2.0 ** (e - 7) * (1 + m / 8)
    return -mag if s else mag


def test_operand_codes_of_plus_and_minus_one(values):
    assert decode_e2m1(values["fp4_plus"]) == 1.0
    assert decode_e2m1(values["fp4_minus"]) == -1.0
    assert decode_e2m1(0) == 0.0
    assert decode_e4m3(values["fp8_plus"]) == 1.0
    assert decode_e4m3(values["fp8_minus"]) == -1.0
    # the unit block scale 0x7F stored in tensor memory: UE8M0 2^(127 - 127)
    assert 2.0 ** (0x7F - 127) == 1.0
    # the decoders themselves: every e2m1 code, and e4m3 extremes
    assert [decode_e2m1(c) for c in range(8)] == [0, 0.5, 1, 1.5, 2, 3, 4, 6]
    assert decode_e4m3(0x7E) == 448.0 and decode_e4m3(0x01) == 2.0 ** -9


def spread(b, nbits, width):
    """Bit k of b (k < nbits) moved to bit width * k."""
    return sum(((b >> k) & 1) << (width * k) for k in range(nbits))


def test_sign_code_bit_spreading(values):
    # every argument below 256; only its low 4 (bytes) or 8 (nibbles) bits count
    for b in range(256):
        assert values[f"spread4_{b}"] == spread(b & 0xF, 4, 8), b
        assert values[f"spread8_{b}"] == spread(b, 8, 4), b
        assert values[f"bmask4_{b}"] == spread(b & 0xF, 4, 8) * 0xFF, b
        assert values[f"nmask8_{b}"] == spread(b, 8, 4) * 0xF, b


def test_sign_codes_of_four_and_eight_spins(values):
    # the one-step epilogue's codes: FP8 byte j = 0x38 | 0x80 for a negative
    # live spin j, 0 for a padded one; FP4 nibble j likewise with 0x2 | 0x8
    for live in range(16):
        for neg in range(16):
            w = values[f"spread4_{live}"] * 0x38 | values[f"spread4_{neg & live}"] << 7
            want = bytes((0xB8 if (neg >> j) & (live >> j) & 1 else 0x38) if (live >> j) & 1
                         else 0 for j in range(4))
            assert w.to_bytes(4, "little") == want
    for live in (0x00, 0xFF, 0x0F, 0xA5, 0x80):
        for neg in (0x00, 0xFF, 0x3C, 0x81):
            w = values[f"spread8_{live}"] * 0x2 | values[f"spread8_{neg & live}"] << 3
            for j in range(8):
                code = (w >> (4 * j)) & 0xF
                want = (0xA if (neg >> j) & 1 else 0x2) if (live >> j) & 1 else 0
                assert code == want


def test_band_order_tile_map(values):
    # t -> (row block, replica block) visits every tile of the grid once
    assert values["tile_map_shapes"] > 1000
    assert values["tile_map_bad"] == 0
    # bands of two replica blocks, the last of one: inside a band the row
    # blocks run in order with the band's replica blocks fastest
    order = [values[f"tile_3_5_2_{t}"] for t in range(15)]
    want = [mb * 5 + rb for band in ((0, 1), (2, 3), (4,)) for mb in range(3) for rb in band]
    assert order == want
