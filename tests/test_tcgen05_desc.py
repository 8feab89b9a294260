"""CPU checks of the tcgen05 descriptor encoders (paper_1802_08557_gb300/csrc/
lp_tcgen05.h) before any of them reaches a GPU: the shared-memory matrix
descriptor and the kind::f16 instruction descriptor, built here field by
field from the PTX ISA bit tables (start, width, meaning) and compared with
the C++ encoders compiled by g++ on the host."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1802_08557_gb300", "csrc")

# (field, first bit, width) of the shared-memory matrix descriptor
SMEM_FIELDS = [("start_addr_4", 0, 14), ("lbo_4", 16, 14), ("sbo_4", 32, 14), ("fixed_001", 46, 3),
               ("base_offset", 49, 3), ("lbo_mode", 52, 1), ("swizzle", 61, 3)]
# (field, first bit, width) of the instruction descriptor for .kind::f16
IDESC_FIELDS = [("sparse_sel", 0, 2), ("sparse", 2, 1), ("saturate", 3, 1), ("d_fmt", 4, 2), ("a_fmt", 7, 3),
                ("b_fmt", 10, 3), ("neg_a", 13, 1), ("neg_b", 14, 1), ("a_major", 15, 1), ("b_major", 16, 1),
                ("n_3", 17, 6), ("m_4", 24, 5), ("max_shift", 30, 2)]


def pack(fields, values):
    word = 0
    for name, lo, width in fields:
        v = values.get(name, 0)
        assert 0 <= v < (1 << width), (name, v)
        word |= v << lo
    return word


def unpack(fields, word):
    return {name: (word >> lo) & ((1 << width) - 1) for name, lo, width in fields}


PROGRAM = r"""
#define __host__
#define __device__
#include <cstdio>
#include "lp_tcgen05.h"
using namespace lpb::tc;
int main() {
    const unsigned addrs[] = {0u, 1024u, 1056u, 33792u, 99328u, 232448u};
    const unsigned sw[] = {kSwizzleNone, kSwizzle128B, kSwizzle64B, kSwizzle32B};
    for (unsigned a : addrs)
        for (unsigned s : sw)
            std::printf("S %u %u %u %u %llu\n", a, 16u, 1024u, s, (unsigned long long)smem_desc(a, 16, 1024, s));
    std::printf("S %u %u %u %u %llu\n", 2048u, 128u, 256u, 0u, (unsigned long long)smem_desc(2048, 128, 256, 0));
    const unsigned ms[] = {64u, 128u}, ns[] = {16u, 64u, 128u, 208u, 256u};
    for (unsigned m : ms)
        for (unsigned n : ns)
            std::printf("I %u %u %u %d\n", m, n, idesc_bf16_f32(m, n), (int)valid_m128_n(n));
    return 0;
}
"""


@pytest.fixture(scope="module")
def encoded(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("tc")
    src = d / "desc.cpp"
    src.write_text(PROGRAM)
    exe = d / "desc"
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-Wall", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    return [line.split() for line in out if line]


def test_smem_descriptor_fields(encoded):
    rows = [r for r in encoded if r[0] == "S"]
    assert len(rows) == 25
    for _, a, lbo, sbo, sw, word in rows:
        a, lbo, sbo, sw, word = int(a), int(lbo), int(sbo), int(sw), int(word)
        want = pack(SMEM_FIELDS, {"start_addr_4": (a >> 4) & 0x3FFF, "lbo_4": lbo >> 4, "sbo_4": sbo >> 4,
                                  "fixed_001": 1, "swizzle": sw})
        assert word == want, (a, lbo, sbo, sw, hex(word), hex(want))
        f = unpack(SMEM_FIELDS, word)
        # nothing outside the documented fields, version 0b001, base offset 0
        assert word & ~pack(SMEM_FIELDS, {n: (1 << w) - 1 for n, _, w in SMEM_FIELDS}) == 0
        assert f["fixed_001"] == 1 and f["base_offset"] == 0 and f["lbo_mode"] == 0


def test_smem_descriptor_k_step_within_a_swizzle_atom(encoded):
    """Advancing the start address by 32 bytes (16 BF16 elements of K) adds 2
    to the encoded start field and changes nothing else."""
    rows = {int(r[1]): int(r[5]) for r in encoded if r[0] == "S" and int(r[4]) == 2}
    assert rows[1056] - rows[1024] == 2
    assert unpack(SMEM_FIELDS, rows[1056])["sbo_4"] == 1024 >> 4


def test_instruction_descriptor_fields(encoded):
    rows = [r for r in encoded if r[0] == "I"]
    assert len(rows) == 10
    for _, m, n, word, valid in rows:
        m, n, word, valid = int(m), int(n), int(word), int(valid)
        want = pack(IDESC_FIELDS, {"d_fmt": 1, "a_fmt": 1, "b_fmt": 1, "n_3": n >> 3, "m_4": m >> 4})
        assert word == want, (m, n, hex(word), hex(want))
        f = unpack(IDESC_FIELDS, word)
        assert f["sparse"] == 0 and f["a_major"] == 0 and f["b_major"] == 0 and f["neg_a"] == 0
        assert valid == int(n % 16 == 0 and 16 <= n <= 256)
    # the kernel's shape: M = 128, N = 128, BF16 x BF16 -> FP32
    assert int([r for r in rows if r[1] == "128" and r[2] == "128"][0][3]) == 0x08200490
