"""The roofline's numerator: bench.py's FP64 instruction counts per primitive equal what
the kernels' own arithmetic (csrc/ddqd.cuh) issues.  The header is compiled for the host
with each FP64 intrinsic counting its calls (every FP64 operation of the primitives goes
through one of them), and the counts of one call of each primitive are compared."""

import os
import shutil
import subprocess

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_1210_0800_gb300", "csrc", "ddqd.cuh")

HOST_INTRINSICS = {
    "__host__ __device__ inline double fma_rn(double a, double b, double c) { return std::fma(a, b, c); }":
        "__host__ __device__ inline double fma_rn(double a, double b, double c) { ++g_fp64; return std::fma(a, b, c); }",
    "__host__ __device__ inline double rcp_rn(double a) { return 1.0 / a; }":
        "__host__ __device__ inline double rcp_rn(double a) { ++g_fp64; return 1.0 / a; }",
    "__host__ __device__ inline double sqrt_rn(double a) { return std::sqrt(a); }":
        "__host__ __device__ inline double sqrt_rn(double a) { ++g_fp64; return std::sqrt(a); }",
    "__host__ __device__ inline double div_rn(double a, double b) { return a / b; }":
        "__host__ __device__ inline double div_rn(double a, double b) { ++g_fp64; return a / b; }",
}

DRIVER = r"""
#include <cstdio>
#include "ddqd.cuh"
namespace mgs { long long g_fp64 = 0; }
using namespace mgs;

template <class Ar>
void count(const char* name, const typename Ar::elem& a, const typename Ar::real& r) {
  const Fp f{1.0, -0.0};
  typename Ar::pacc p;
  typename Ar::elem q = a;
  long long mac = 0, upd = 0, norm = 0, div = 0;
  for (int part = 0; part < 2; ++part) {
    Ar::pzero(p);
    g_fp64 = 0; Ar::mac_part(f, p, a, a, part); mac += g_fp64;
    g_fp64 = 0; Ar::update_part(f, q, a, a, part); upd += g_fp64;
  }
  Ar::pzero(p);
  g_fp64 = 0; Ar::mac_part(f, p, a, a, 0); norm = g_fp64;  // |x|^2: the real part alone
  g_fp64 = 0;
  const double inv = Ar::inv_lead(r);
  Ar::div_real_part(f, q, a, r, inv, 0);
  Ar::div_real_part(f, q, a, r, inv, 1);
  div = g_fp64;
  std::printf("%s %lld %lld %lld %lld\n", name, mac, upd, norm, div);
}

int main() {
  count<D>("1", D::elem{{1.0, 2.0}}, D::real{3.0});
  count<DD>("2", DD::elem{{1.0, 1e-17, 2.0, 2e-17}}, DD::real{3.0, 3e-17});
  count<QD>("4", QD::elem{{1.0, 1e-17, 1e-34, 1e-51, 2.0, 2e-17, 2e-34, 2e-51}}, QD::real{{3.0, 3e-17, 3e-34, 3e-51}});
  return 0;
}
"""


def test_bench_counts_match_the_arithmetic(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    src = open(HEADER).read()
    for old, new in HOST_INTRINSICS.items():
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    src = src.replace("namespace mgs {", "namespace mgs {\nextern long long g_fp64;", 1)
    (tmp_path / "ddqd.cuh").write_text(src)
    (tmp_path / "count.cpp").write_text(DRIVER)
    exe = tmp_path / "count"
    subprocess.check_call([gxx, "-O1", "-std=c++17", "-Wno-unknown-pragmas", "-o", str(exe), str(tmp_path / "count.cpp")])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {}
    for line in out:
        if line.strip():
            L, mac, upd, norm, div = line.split()
            got[int(L)] = dict(mac=int(mac), upd=int(upd), norm=int(norm), div=int(div))
    assert got == bench.COST
