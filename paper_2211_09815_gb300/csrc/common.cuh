// Shared device helpers for the particle-mesh kernels: complex arithmetic on
// float2/double2, the deterministic fixed-point conventions, and small indexing helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pmgb {

template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };
template <typename T> using cx_t = typename Cx<T>::type;

template <typename C> __device__ __forceinline__ C cmake(decltype(C{}.x) re, decltype(C{}.x) im) {
  C r; r.x = re; r.y = im; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmake<C>(a.x, -a.y); }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return cmake<C>(a.x * s, a.y * s); }
// multiply by i
template <typename C> __device__ __forceinline__ C cmul_i(C a) { return cmake<C>(-a.y, a.x); }

// Integer <-> float conversions of the fixed-point accumulators on the integer ALU
// (correctly rounded, nearest-even): the hardware conversions involving 64-bit integers go
// through the FP64 pipe, which is slow on this part.
__device__ __forceinline__ float ll2f_rn(long long a) {
  if (a == 0) return 0.0f;
  const unsigned long long ua = a < 0 ? 0ull - (unsigned long long)a : (unsigned long long)a;
  const int lz = __clzll(ua);
  const unsigned long long m = ua << lz;                 // leading one at bit 63
  unsigned mant = (unsigned)(m >> 40);                   // 24 significant bits
  const unsigned long long rest = m & 0xFFFFFFFFFFull;    // the 40 bits shifted out
  if (rest > 0x8000000000ull || (rest == 0x8000000000ull && (mant & 1u))) ++mant;
  int e = 63 - lz + 127;
  if (mant == (1u << 24)) {
    mant >>= 1;
    ++e;
  }
  return __uint_as_float(((unsigned)e << 23) | (mant & 0x7FFFFFu) | (a < 0 ? 0x80000000u : 0u));
}
// |v| < 2^62
__device__ __forceinline__ long long f2ll_rn(float v) {
  const unsigned b = __float_as_uint(v);
  const int e = (int)((b >> 23) & 0xFFu);
  if (e < 126) return 0;                                 // |v| < 0.5
  const unsigned long long mant = (b & 0x7FFFFFu) | 0x800000u;
  const int sh = e - 150;                                // v = mant * 2^sh
  unsigned long long r;
  if (sh >= 0) {
    r = mant << sh;
  } else {
    const int rs = -sh;                                  // 1..24
    r = mant >> rs;
    const unsigned long long rem = mant & ((1ull << rs) - 1), half = 1ull << (rs - 1);
    if (rem > half || (rem == half && (r & 1ull))) ++r;
  }
  return (b >> 31) ? -(long long)r : (long long)r;
}

// 2^e built from its bit pattern, for e in the normal range of T (the FP64 pipe that
// ldexp goes through is slow on this part)
template <typename T> __device__ __forceinline__ T pow2i(int e);
template <> __device__ __forceinline__ float pow2i<float>(int e) { return __int_as_float((e + 127) << 23); }
template <> __device__ __forceinline__ double pow2i<double>(int e) {
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// four reals of one mesh cell (force components and the adjoint potential), one load
template <typename T> struct alignas(4 * sizeof(T)) V4 { T x, y, z, w; };

// Layout of one complex half spectrum of an n^3 real mesh ("spectrum buffer"):
//   main:  [n][n][n/2] complex, kx = 0..n/2-1 along the fastest axis
//   side:  [n][n] complex, the kx = n/2 (Nyquist) plane
// main + side hold n^3 + 2 n^2 reals, the real mesh [n][n][n] lives at the start of the
// same buffer after an inverse transform.  Instances of a batch follow each other.
__host__ __device__ inline long long spec_main_len(int n) { return (long long)n * n * (n / 2); }
__host__ __device__ inline long long spec_len_cx(int n) { return spec_main_len(n) + (long long)n * n; }

// z blocking of the main part of the mesh spectra: row (z, y) of the main array is stored
// at ((z / zb) n + y) zb + z mod zb.  With zb = 1 this is the plain [z][y] order; for
// 1024^3 meshes (zb = 8) a column tile of the y pass spans 32 MB instead of 4 MB and one
// of the z pass 128 address blocks of 32 KB instead of 1024 rows 4 MB apart, which keeps
// the pages a tile touches (and its address translations) few.  Lattice spectra and the
// side planes always use the plain order.
__host__ __device__ constexpr int spec_zb(int n) { return n >= 1024 ? 8 : 1; }
__host__ __device__ constexpr int spec_lzb(int n) { return n >= 1024 ? 3 : 0; }   // log2 spec_zb
// row of (z, y) with blocks of 2^lzb z values (shifts: the x passes are integer bound)
__host__ __device__ inline long long spec_row(int n, int lzb, int z, int y) {
  return ((((long long)(z >> lzb) * n + y)) << lzb) | (z & ((1 << lzb) - 1));
}

// Element q of a small array held in kernel parameters, chosen with selects: a dynamic
// index into the parameter block would copy it to local memory in every thread.
template <typename X, int K>
__device__ __forceinline__ X pick(const X (&a)[K], int q) {
  X r = a[0];
#pragma unroll
  for (int i = 1; i < K; ++i)
    if (q == i) r = a[i];
  return r;
}

// signed frequency of index i on an axis of length n, in [-n/2, n/2)
__device__ __forceinline__ int freq_of(int i, int n) { return i < n / 2 ? i : i - n; }

}  // namespace pmgb
