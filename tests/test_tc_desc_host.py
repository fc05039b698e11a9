"""Field-by-field check of the tcgen05 descriptors the tensor-core product
builds (csrc/tc_desc.h), on the host with no GPU.

The header is compiled with g++ into a tiny program that prints the 64-bit
shared-memory descriptors and 32-bit instruction descriptors the kernel
uses; each field is then decoded here from the bit positions of NVIDIA's
public PTX ISA tables and compared with the value the kernel needs: a wrong
shift or mask in the header (a field that lands one bit off) fails here
instead of on the device.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1812_07167_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include "tc_desc.h"
int main() {
  const unsigned addrs[] = {0u, 1024u, 1024u + 32u, 65536u + 96u, 196608u + 49152u};
  for (unsigned a : addrs)
    std::printf("S %u %llu\n", a, (unsigned long long)hps::tc::smem_desc_sw128_kmajor(a));
  const int shapes[][2] = {{128, 128}, {128, 64}, {64, 256}, {128, 256}};
  for (auto &s : shapes)
    for (int neg = 0; neg < 2; neg++)
      std::printf("I %d %d %d %u\n", s[0], s[1], neg, hps::tc::idesc_bf16_f32(s[0], s[1], neg != 0));
  return 0;
}
"""


def bits(v, lo, hi):
    """Bits lo .. hi - 1 of v."""
    return (v >> lo) & ((1 << (hi - lo)) - 1)


@pytest.fixture(scope="module")
def printed(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("tcdesc")
    src = d / "t.cpp"
    src.write_text(PROG)
    exe = d / "t"
    subprocess.run([gxx, "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    return [line.split() for line in out if line]


def test_shared_memory_descriptor_fields(printed):
    seen = 0
    for row in printed:
        if row[0] != "S":
            continue
        addr, d = int(row[1]), int(row[2])
        assert bits(d, 0, 14) == (addr >> 4) & 0x3FFF      # start address >> 4
        assert bits(d, 14, 16) == 0
        assert bits(d, 16, 30) == 1                         # leading offset: unused, 16 B
        assert bits(d, 30, 32) == 0
        assert bits(d, 32, 46) == 1024 >> 4                 # 8 rows of 128 bytes between row groups
        assert bits(d, 46, 49) == 0b001                     # fixed constant of the sm_100 format
        assert bits(d, 49, 52) == 0                         # base offset: 1 KB aligned atoms
        assert bits(d, 52, 53) == 0                         # relative leading offset
        assert bits(d, 53, 61) == 0
        assert bits(d, 61, 64) == 2                         # 128-byte swizzle
        seen += 1
    assert seen == 5


def test_k_steps_move_the_start_address_by_32_bytes(printed):
    # the kernel advances K by 16 bf16 inside a 128-byte swizzled row: +32 B
    d = {int(r[1]): int(r[2]) for r in printed if r[0] == "S"}
    assert bits(d[1024 + 32], 0, 14) - bits(d[1024], 0, 14) == 2
    assert d[1024 + 32] - d[1024] == 2


def test_instruction_descriptor_fields(printed):
    seen = 0
    for row in printed:
        if row[0] != "I":
            continue
        M, N, neg, d = int(row[1]), int(row[2]), int(row[3]), int(row[4])
        assert d < (1 << 32)
        assert bits(d, 0, 2) == 0      # sparsity selector
        assert bits(d, 2, 3) == 0      # dense
        assert bits(d, 3, 4) == 0      # no saturation
        assert bits(d, 4, 6) == 1      # D in f32
        assert bits(d, 6, 7) == 0
        assert bits(d, 7, 10) == 1     # A bf16
        assert bits(d, 10, 13) == 1    # B bf16
        assert bits(d, 13, 14) == neg  # negate A
        assert bits(d, 14, 15) == 0    # B not negated
        assert bits(d, 15, 16) == 0    # A K-major
        assert bits(d, 16, 17) == 0    # B K-major
        assert bits(d, 17, 23) == N // 8
        assert bits(d, 23, 24) == 0
        assert bits(d, 24, 29) == M // 16
        assert bits(d, 29, 32) == 0
        seen += 1
    assert seen == 8


def test_kernel_shapes_are_valid_tcgen05_shapes(printed):
    # cta_group::1, kind::f16: M in {64, 128}; N a multiple of 16 (M = 128)
    # or 8 (M = 64) in [16, 256]; the kernel uses M = 128 with N = 128 and 64
    for M, N in ((128, 128), (128, 64)):
        assert M in (64, 128) and N % 16 == 0 and 16 <= N <= 256
