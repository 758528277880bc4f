// Hand-written batched 3-D real FFT for the particle-mesh force (Sec. 2.2, Eq. 11):
// kernels and launchers, templated on the real type.  Included once per precision.
//
// Spectrum layout (see common.cuh): main [n][n][n/2] complex + side [n][n] complex
// (kx = n/2) per instance.  Forward R2C = x pass (rows, real -> half spectrum, packing
// two reals per complex and splitting even/odd afterwards) then y and z column passes.
// The inverse runs z, y, then the x pass (C2R).  Transforms are unnormalised both ways;
// the 1/n^3 of the inverse is folded into the Fourier multipliers.
#pragma once
#include <type_traits>

#include <cuda_fp16.h>

#include "fft.cuh"
#include "fft_tma.cuh"
#include "pm_internal.h"

namespace pmgb {

// ---------------------------------------------------------------- column passes
__device__ __forceinline__ long long seq_base(const SeqMap& m, int s) {
  const int col = s % m.ncols;
  const int t = s / m.ncols;
  const int o0 = t % m.n0;
  const int o1 = t / m.n0;
  return (long long)o1 * m.os1 + (long long)o0 * m.os0 + (long long)col * m.cs;
}

template <typename T, int L, int DIR>
__global__ void __launch_bounds__(ColTile<T, L>::NT, 2)
k_fft_cols(const SeqMap mm, const SeqMap ms, int ntiles_main, ColBufs<T> bufs,
           const cx_t<T>* __restrict__ tw) {
  using C = cx_t<T>;
  using TL = ColTile<T, L>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const bool side = blockIdx.x >= (unsigned)ntiles_main;
  const SeqMap& m = side ? ms : mm;
  const int s0 = (side ? blockIdx.x - ntiles_main : blockIdx.x) * TL::TC;
  const int s = s0 + threadIdx.x % TL::TC;
  const bool valid = s < m.nseq;
  C* base = pick(bufs.p, blockIdx.y) + (valid ? seq_base(m, s) : 0);
  GlobalSeq<C> g{base, m.es, valid};
  SmemTile<C, TL::LD> t{sm};
  fft_tile<T, L, TL::TC, TL::NT, DIR>(g, t, g, tw);
}

// y passes of the separable force components (sequences of mm/ms as in k_fft_cols; the
// side plane kx = n/2 has k_2 = 0 by the Nyquist rule, main columns have k_2 = kx = col).
// Split (inverse): U -> out1 = IFFT(U), U <- IFFT(-i k_1 U).
// Merge (forward): P_1 <- i (k_1 FFT(P_1) + k_2 FFT(P_2)).
template <typename T, int N>
struct GSeqNegIK {   // -i k_row v read from a global sequence
  const cx_t<T>* p;
  long long es;
  bool valid;
  __device__ __forceinline__ cx_t<T> ld(int row, int) const {
    if (!valid) return cmake<cx_t<T>>(0, 0);
    const cx_t<T> v = p[(long long)row * es];
    const T s = (T)fc_row<N>(row);
    return cmake<cx_t<T>>(v.y * s, -v.x * s);
  }
};
template <typename T, int N, int LD>
struct SAccIK {      // A = i k_row v into a shared tile
  cx_t<T>* p;
  __device__ __forceinline__ void st(int row, int c, cx_t<T> v) const {
    const T s = (T)fc_row<N>(row);
    p[srow(row) * LD + c] = cmake<cx_t<T>>(-v.y * s, v.x * s);
  }
};
template <typename T, int LD>
struct GMergeIK {    // out = A + i k2 v
  const cx_t<T>* acc;
  cx_t<T>* out;
  long long es;
  bool valid;
  T k2;
  __device__ __forceinline__ void st(int row, int c, cx_t<T> v) const {
    if (!valid) return;
    const cx_t<T> a = acc[srow(row) * LD + c];
    out[(long long)row * es] = cmake<cx_t<T>>(a.x - v.y * k2, a.y + v.x * k2);
  }
};

template <typename T, int L, int MODE>   // MODE 1: split, 2: merge
__global__ void __launch_bounds__(ColTile<T, L>::NT, 1)
k_fft_cols_yx(const SeqMap mm, const SeqMap ms, int ntiles_main, ColBufs<T> bufs,
              const cx_t<T>* __restrict__ tw) {
  using C = cx_t<T>;
  using TL = ColTile<T, L>;
  constexpr int TILE = skew_rows(L) * TL::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* A = reinterpret_cast<C*>(smem_raw);
  C* B = A + TILE;
  const bool side = blockIdx.x >= (unsigned)ntiles_main;
  const SeqMap& m = side ? ms : mm;
  const int s0 = (side ? blockIdx.x - ntiles_main : blockIdx.x) * TL::TC;
  const int s = s0 + threadIdx.x % TL::TC;
  const bool valid = s < m.nseq;
  const long long off = valid ? seq_base(m, s) : 0;
  SmemTile<C, TL::LD> ta{A};
  if constexpr (MODE == 1) {
    GlobalSeq<C> gu{bufs.p[0] + off, m.es, valid};
    GlobalSeq<C> g1{bufs.p[1] + off, m.es, valid};
    fft_tile<T, L, TL::TC, TL::NT, +1>(gu, ta, g1, tw);
    __syncthreads();
    GSeqNegIK<T, L> src{bufs.p[0] + off, m.es, valid};
    fft_tile<T, L, TL::TC, TL::NT, +1>(src, ta, gu, tw);
  } else {
    GlobalSeq<C> g1{bufs.p[0] + off, m.es, valid};
    GlobalSeq<C> g2{bufs.p[1] + off, m.es, valid};
    SAccIK<T, L, TL::LD> acc{B};
    fft_tile<T, L, TL::TC, TL::NT, -1>(g1, ta, acc, tw);
    __syncthreads();
    const T k2 = side ? (T)0 : (T)(s % m.ncols);
    GMergeIK<T, TL::LD> dst{B, bufs.p[0] + off, m.es, valid, k2};
    fft_tile<T, L, TL::TC, TL::NT, -1>(g2, ta, dst, tw);
  }
}

// ---------------------------------------------------------------- x pass, R2C
// rows of n = 2L reals -> L complex (main) + 1 (side).  The row pairs (2j, 2j+1) are read
// as one complex number and transformed as L-point sequences; the even/odd split below
// recovers the real transform.  The buffers of one row tile are neighbouring blocks.
//
// Work items of the split (and of the untangling before the C2R below) are the pairs
// (k, L - k), k < L/2, of every row, indexed row-major so that a power of two divides them,
// and then the middle k = L/2 of every row; the address of each row of the tile is worked
// out once, into shared memory.
template <typename T, int L>
__global__ void __launch_bounds__(RowTile<T, L>::NT)
k_fft_x_r2c(RowJob<T> job, int nrows, int nbuf, const cx_t<T>* __restrict__ twL,
            const cx_t<T>* __restrict__ twN) {
  using C = cx_t<T>;
  using TL = RowTile<T, L>;
  constexpr int N = 2 * L;
  constexpr int RT = TL::TR;   // rows per tile
  constexpr int KH = L / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ C* s_out[RT];     // main spectrum row of each tile row (null past nrows)
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int qb = blockIdx.x % nbuf;
  const int r0 = (blockIdx.x / nbuf) * RT;
  const long long rows_per_inst = (long long)N * N;
  // all rows of a tile belong to one instance (RT divides N^2) and are consecutive there
  const int inst0 = (int)(min((long long)r0, (long long)nrows - 1) / rows_per_inst);
  const long long rr0 = r0 % rows_per_inst;
  const RowBuf<T> rb0 = pick(job.b, qb);
  C* const spec0 = rb0.spec + inst0 * spec_len_cx(N);
  for (int c = threadIdx.x; c < RT; c += TL::NT) {
    const long long rr = rr0 + c;
    s_out[c] = r0 + c < nrows ? spec0 + spec_row(N, job.lzb, (int)(rr / N), (int)(rr % N)) * L : nullptr;
  }
  // load, transposing into [L][LD]; every load of the thread is issued before the first
  // shared-memory store so that ITER loads per thread are in flight at once.  The tile's
  // rows are one contiguous run of RT n reals.
  constexpr int ITER = RT * L / TL::NT;
  static_assert(ITER * TL::NT == RT * L, "row loads must divide evenly");
  const C* tile_in = reinterpret_cast<const C*>(reinterpret_cast<const T*>(rb0.real) + inst0 * rb0.real_is + rr0 * N);
  C raw[ITER];
#pragma unroll
  for (int it = 0; it < ITER; ++it) {
    const int idx = threadIdx.x + it * TL::NT;
    raw[it] = r0 + idx / L < nrows ? tile_in[idx] : cmake<C>(0, 0);
  }
#pragma unroll
  for (int it = 0; it < ITER; ++it) {
    const int idx = threadIdx.x + it * TL::NT;
    const int row = idx / L, j = idx % L;
    sm[srow(j) * TL::LD + row] = raw[it];
  }
  __syncthreads();
  SmemTile<C, TL::LD> t{sm};
  fft_tile<T, L, TL::TR, TL::NT, -1, typename TL::P>(t, t, t, twL);
  __syncthreads();
  // even/odd split: X[k] = E[k] + W^k O[k], E = (Z[k] + conj Z[L-k]) / 2, O = -i (Z[k] - conj Z[L-k]) / 2
  constexpr int PAIRS = RT * KH;
  for (int u = threadIdx.x; u < PAIRS + RT; u += TL::NT) {
    const int c = u < PAIRS ? u / KH : u - PAIRS;
    const int k = u < PAIRS ? u % KH : KH;
    C* out = s_out[c];
    if (!out) continue;
    const C zk = sm[srow(k) * TL::LD + c];
    if (k == 0) {
      out[0] = cmake<C>(zk.x + zk.y, (T)0);
      spec0[spec_main_len(N) + rr0 + c] = cmake<C>(zk.x - zk.y, (T)0);
      continue;
    }
    const C zm = sm[srow(L - k) * TL::LD + c];
    const T h = (T)0.5;
    const C e = cscale(cadd(zk, cconj(zm)), h);
    const C d = cscale(csub(zk, cconj(zm)), h);
    const C o = cmake<C>(d.y, -d.x);  // -i d
    const C w = __ldg(twN + k);       // exp(-2 pi i k / N)
    const C wo = cmul(w, o);
    out[k] = cadd(e, wo);
    if (k != L - k) out[L - k] = cconj(csub(e, wo));
  }
}

// ---------------------------------------------------------------- x pass, C2R
// L complex (main) + side -> n = 2L reals (unnormalised).  The output may alias the input.
// Z[k] = E'[k] + i O'[k], E' = X[k] + conj X[L-k], O' = (X[k] - conj X[L-k]) conj(W^k), for
// the pairs (k, L - k) of every row (work items as in the R2C split).
template <typename T, int L, int TR, int NT>
struct C2RUntangle {
  static constexpr int KH = L / 2;
  static constexpr int PAIRS = TR * KH;
  static constexpr int ITEMS = PAIRS + TR;                    // + the middle k = L/2 of every row
  static constexpr int ITER = (ITEMS + NT - 1) / NT;
  __device__ __forceinline__ static int seq(int u) { return u < PAIRS ? u / KH : u - PAIRS; }
  __device__ __forceinline__ static int freq(int u) { return u < PAIRS ? u % KH : KH; }
};

template <typename T, int L>
__global__ void __launch_bounds__(RowTile<T, L>::NT)
k_fft_x_c2r(RowJob<T> job, int nrows, const cx_t<T>* __restrict__ twL, const cx_t<T>* __restrict__ twN) {
  using C = cx_t<T>;
  using TL = RowTile<T, L>;
  using U = C2RUntangle<T, L, TL::TR, TL::NT>;
  constexpr int N = 2 * L;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ const C* s_in[TL::TR];     // main spectrum row of each tile row (null past nrows)
  C* sm = reinterpret_cast<C*>(smem_raw);
  const RowBuf<T> rb = pick(job.b, blockIdx.y);
  const int r0 = blockIdx.x * TL::TR;
  const long long rows_per_inst = (long long)N * N;
  // all rows of a tile belong to one instance (TR divides N^2) and are consecutive there
  const int inst0 = (int)(min((long long)r0, (long long)nrows - 1) / rows_per_inst);
  const long long rr0 = r0 % rows_per_inst;
  const C* const base = rb.spec + inst0 * spec_len_cx(N);
  for (int c = threadIdx.x; c < TL::TR; c += TL::NT) {
    const long long rr = rr0 + c;
    s_in[c] = r0 + c < nrows ? base + spec_row(N, job.lzb, (int)(rr / N), (int)(rr % N)) * L : nullptr;
  }
  __syncthreads();
  // all loads of the thread are issued before the first use
  C xk[U::ITER], xm[U::ITER];
#pragma unroll
  for (int it = 0; it < U::ITER; ++it) {
    const int u = threadIdx.x + it * TL::NT;
    xk[it] = cmake<C>(0, 0);
    xm[it] = cmake<C>(0, 0);
    if (u < U::ITEMS) {
      const int c = U::seq(u), k = U::freq(u);
      const C* in = s_in[c];
      if (in) {
        xk[it] = in[k];
        xm[it] = k == 0 ? base[spec_main_len(N) + rr0 + c] : in[L - k];
      }
    }
  }
#pragma unroll
  for (int it = 0; it < U::ITER; ++it) {
    const int u = threadIdx.x + it * TL::NT;
    if (u >= U::ITEMS) continue;
    const int row = U::seq(u), k = U::freq(u);
    C zk, zm = cmake<C>(0, 0);
    if (k == 0) {
      const T x0 = xk[it].x, xl = xm[it].x;
      zk = cmake<C>(x0 + xl, x0 - xl);
    } else {
      const C e = cadd(xk[it], cconj(xm[it]));
      const C d = csub(xk[it], cconj(xm[it]));
      const C o = cmul(d, cconj(__ldg(twN + k)));
      zk = cadd(e, cmul_i(o));
      zm = cadd(cconj(e), cmul_i(cconj(o)));
    }
    sm[srow(k) * TL::LD + row] = zk;
    if (k != 0 && k != L - k) sm[srow(L - k) * TL::LD + row] = zm;
  }
  __syncthreads();
  SmemTile<C, TL::LD> t{sm};
  fft_tile<T, L, TL::TR, TL::NT, +1, typename TL::P>(t, t, t, twL);
  __syncthreads();
  // the tile's rows are one contiguous run of TR n reals
  C* tile_out = reinterpret_cast<C*>(reinterpret_cast<T*>(rb.real) + inst0 * rb.real_is + rr0 * N);
  for (int idx = threadIdx.x; idx < TL::TR * L; idx += TL::NT) {
    const int row = idx / L, j = idx % L;
    if (r0 + row >= nrows) continue;
    tile_out[idx] = sm[srow(j) * TL::LD + row];
  }
}

// C2R x pass of four components at once, writing one V4 per cell ([cell](c0, c1, c2, c3),
// instances back to back) so that a gather reads all components of a corner with one
// load.  The block holds TR/4 rows of each component; a null spectrum pointer reads as 0.
// Component dq (or none if dq < 0) is multiplied by -i k_x on the way in.
template <typename T, int L, int Q> struct C2R4Tile {
  using P = typename RowTile<T, L>::P;
  static constexpr int RT = RowTile<T, L>::TR / 4;       // rows per block
  static constexpr int TR = Q * RT;                      // sequences per block
  // above 256 threads, two radix items per thread (measured faster at L = 512)
  static constexpr int NT0 = TR * L / P::RMAX;
  static constexpr int NT = (NT0 > 256 && (NT0 / 2) % 32 == 0) ? NT0 / 2 : NT0;
  static constexpr int LD = TR + 1;
  static constexpr int SMEM = skew_rows(L) * LD * (int)sizeof(cx_t<T>);
};

// H: the FP16 force mesh (pm_config.half_force, FP32 only): per cell four halves, each
// field of a row scaled by 2^-e so that the row's largest magnitude lies in [2^14, 2^15),
// e stored as one int8 per (row, field) in fexp ([rows][4]); FP16 keeps 11 significant
// bits of every value in the row down to 2^-29 of its largest.
template <typename T, int L, int Q, bool H = false>
__global__ void __launch_bounds__(C2R4Tile<T, L, Q>::NT)
k_fft_x_c2r4(RowJob<T> job, int nrows, int dq, void* __restrict__ out, signed char* __restrict__ fexp,
             const cx_t<T>* __restrict__ twL, const cx_t<T>* __restrict__ twN) {
  using C = cx_t<T>;
  using TL = C2R4Tile<T, L, Q>;
  using U = C2RUntangle<T, L, TL::TR, TL::NT>;
  constexpr int N = 2 * L;
  constexpr int RT = TL::RT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ const C* s_in[TL::TR];     // main spectrum row of sequence c = (component, row)
  __shared__ const C* s_side[TL::TR];   // its side-plane element (kx = L)
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int r0 = blockIdx.x * RT;
  const long long rows_per_inst = (long long)N * N;
  for (int c = threadIdx.x; c < TL::TR; c += TL::NT) {
    const int q = c / RT, grow = r0 + c % RT;
    const C* in = nullptr;
    const C* side = nullptr;
    if (grow < nrows) {
      const C* base = pick(job.b, q).spec + (grow / rows_per_inst) * spec_len_cx(N);
      const long long rr = grow % rows_per_inst;
      in = base + spec_row(N, job.lzb, (int)(rr / N), (int)(rr % N)) * L;
      side = base + spec_main_len(N) + rr;
    }
    s_in[c] = in;
    s_side[c] = side;
  }
  __syncthreads();
  C xk[U::ITER], xm[U::ITER];
#pragma unroll
  for (int it = 0; it < U::ITER; ++it) {
    const int u = threadIdx.x + it * TL::NT;
    xk[it] = cmake<C>(0, 0);
    xm[it] = cmake<C>(0, 0);
    if (u < U::ITEMS) {
      const int c = U::seq(u), k = U::freq(u);
      const C* in = s_in[c];
      if (in) {
        xk[it] = in[k];
        xm[it] = k == 0 ? *s_side[c] : in[L - k];
      }
    }
  }
#pragma unroll
  for (int it = 0; it < U::ITER; ++it) {
    const int u = threadIdx.x + it * TL::NT;
    if (u >= U::ITEMS) continue;
    const int c = U::seq(u), k = U::freq(u);
    if (c / RT == dq) {
      // component dq is the x derivative -i k_x of its spectrum (Nyquist kx = L: 0)
      const T sk = (T)k, sl = k == 0 ? (T)0 : (T)(L - k);
      xk[it] = cmake<C>(xk[it].y * sk, -xk[it].x * sk);
      xm[it] = cmake<C>(xm[it].y * sl, -xm[it].x * sl);
    }
    C zk, zm = cmake<C>(0, 0);
    if (k == 0) {
      const T x0 = xk[it].x, xl = xm[it].x;
      zk = cmake<C>(x0 + xl, x0 - xl);
    } else {
      const C e = cadd(xk[it], cconj(xm[it]));
      const C d = csub(xk[it], cconj(xm[it]));
      const C o = cmul(d, cconj(__ldg(twN + k)));
      zk = cadd(e, cmul_i(o));
      zm = cadd(cconj(e), cmul_i(cconj(o)));
    }
    sm[srow(k) * TL::LD + c] = zk;
    if (k != 0 && k != L - k) sm[srow(L - k) * TL::LD + c] = zm;
  }
  __syncthreads();
  SmemTile<C, TL::LD> t{sm};
  fft_tile<T, L, TL::TR, TL::NT, +1, typename TL::P>(t, t, t, twL);
  __syncthreads();
  if constexpr (!H) {
    V4<T>* const tile_out = reinterpret_cast<V4<T>*>(out) + (long long)r0 * N;
    for (int idx = threadIdx.x; idx < RT * L; idx += TL::NT) {
      const int row = idx / L, j = idx % L;
      if (r0 + row >= nrows) continue;
      const C v0 = sm[srow(j) * TL::LD + row], v1 = sm[srow(j) * TL::LD + RT + row];
      const C v2 = sm[srow(j) * TL::LD + 2 * RT + row];
      const C v3 = Q == 4 ? sm[srow(j) * TL::LD + (Q - 1) * RT + row] : cmake<C>(0, 0);
      V4<T>* o = tile_out + 2 * idx;
      o[0] = V4<T>{v0.x, v1.x, v2.x, v3.x};
      o[1] = V4<T>{v0.y, v1.y, v2.y, v3.y};
    }
  } else {
    static_assert(sizeof(T) == 4, "the FP16 force mesh is an FP32-path form");
    // largest magnitude per (row, field): bit patterns of non-negative floats order like
    // the values, so an unsigned max finds it
    __shared__ unsigned smax[RT * 4];
    __shared__ float sscale[RT * 4];
    for (int k = threadIdx.x; k < RT * 4; k += TL::NT) smax[k] = 0u;
    __syncthreads();
    // with L and NT multiples of 32, a warp's 32 items lie in one sequence and every lane
    // runs the same iterations: one reduction and one atomic per warp
    for (int k = threadIdx.x; k < Q * RT * L; k += TL::NT) {
      const int c = k / L, j = k % L;   // sequence c = q RT + row
      const C v = sm[srow(j) * TL::LD + c];
      unsigned m = __float_as_uint(fmaxf(fabsf(v.x), fabsf(v.y)));
      if constexpr (L % 32 == 0 && TL::NT % 32 == 0) {
        m = __reduce_max_sync(0xFFFFFFFFu, m);
        if ((threadIdx.x & 31) == 0) atomicMax(&smax[(c % RT) * 4 + c / RT], m);
      } else {
        atomicMax(&smax[(c % RT) * 4 + c / RT], m);
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < RT * 4; k += TL::NT) {
      const float m = __uint_as_float(smax[k]);
      int e = m > 0.f ? ilogbf(m) - 14 : 0;   // m 2^-e in [2^14, 2^15)
      e = e < -120 ? -120 : (e > 120 ? 120 : e);
      sscale[k] = __int_as_float((127 - e) << 23);   // 2^-e
      const int row = k / 4;
      if (r0 + row < nrows) fexp[(long long)(r0 + row) * 4 + k % 4] = (signed char)e;
    }
    __syncthreads();
    uint4* const tile_out = reinterpret_cast<uint4*>(out) + (long long)r0 * (N / 2);
    for (int idx = threadIdx.x; idx < RT * L; idx += TL::NT) {
      const int row = idx / L, j = idx % L;
      if (r0 + row >= nrows) continue;
      const float* sc = sscale + row * 4;
      const C v0 = sm[srow(j) * TL::LD + row], v1 = sm[srow(j) * TL::LD + RT + row];
      const C v2 = sm[srow(j) * TL::LD + 2 * RT + row];
      const C v3 = Q == 4 ? sm[srow(j) * TL::LD + (Q - 1) * RT + row] : cmake<C>(0, 0);
      // cells 2j and 2j + 1 of the row: (f_0, f_1, f_2, f_3) as two half2 each
      const __half2 a0 = __floats2half2_rn(v0.x * sc[0], v1.x * sc[1]), a1 = __floats2half2_rn(v2.x * sc[2], v3.x * sc[3]);
      const __half2 b0 = __floats2half2_rn(v0.y * sc[0], v1.y * sc[1]), b1 = __floats2half2_rn(v2.y * sc[2], v3.y * sc[3]);
      tile_out[idx] = make_uint4(*reinterpret_cast<const unsigned*>(&a0), *reinterpret_cast<const unsigned*>(&a1),
                                 *reinterpret_cast<const unsigned*>(&b0), *reinterpret_cast<const unsigned*>(&b1));
    }
  }
}

// ---------------------------------------------------------------- fused z passes
// Sequence s of a z pass: main tiles s -> (b, y, kx), side tiles s -> (b, y) with kx = n/2.
struct ZSeq {
  int b, f1, f2;      // instance, signed y frequency, x frequency (0..n/2)
  long long base;     // complex offset of element kz = 0
  long long es;       // complex stride along z
  bool valid;
};
template <int N>
__device__ __forceinline__ ZSeq zseq(int s, bool side, int batch) {
  ZSeq q;
  if (!side) {
    const int kx = s % (N / 2), t = s / (N / 2);
    const int y = t % N;
    q.b = t / N;
    q.f1 = freq_of(y, N);
    q.f2 = kx;
    q.base = q.b * spec_len_cx(N) + (long long)y * (N / 2) + kx;
    q.es = (long long)N * (N / 2);
  } else {
    const int y = s % N;
    q.b = s / N;
    q.f1 = freq_of(y, N);
    q.f2 = N / 2;
    q.base = q.b * spec_len_cx(N) + spec_main_len(N) + y;
    q.es = N;
  }
  q.valid = q.b < batch;
  if (!q.valid) q.b = 0;
  return q;
}

// multiplier data for one sequence: g(f0) = coef * d12 * dtab[f0] / (f0^2 + n12)
template <typename T>
struct GreenSeq {
  T coef, d12;
  int n12, f1, f2;
  const T* dtab;
  int n;
  __device__ __forceinline__ T g(int f0) const {
    const int n2 = f0 * f0 + n12;
    if (n2 == 0) return (T)0;
    T v = coef * d12 / (T)n2;
    if (dtab) v *= dtab[f0 < 0 ? f0 + n : f0];
    return v;
  }
  // k_c / kf for component c with the Nyquist plane of axis c zeroed
  __device__ __forceinline__ int fc(int comp, int f0) const {
    if (comp == 0) return f0 == -n / 2 ? 0 : f0;
    if (comp == 1) return f1 == -n / 2 ? 0 : f1;
    return f2 == n / 2 ? 0 : f2;
  }
};

// Source of an inverse z stage in the force pass, output `mode`: 0: -i k_0 G v (z force),
// 1: G v (shared by the y and x force components, whose -i k_1, -i k_2 are constant along
// a z column and are applied in the y and x passes)
template <typename T, int LD>
struct MulSrc {
  const cx_t<T>* p;
  GreenSeq<T> gs;
  int mode;
  __device__ __forceinline__ cx_t<T> ld(int row, int c) const {
    using C = cx_t<T>;
    const C v = p[srow(row) * LD + c];
    const int f0 = freq_of(row, gs.n);
    const T g = gs.g(f0);
    if (mode == 1) return cmake<C>(v.x * g, v.y * g);
    const T s = (T)gs.fc(0, f0) * g;
    return cmake<C>(v.y * s, -v.x * s);
  }
};

// Destination of a forward z stage in the adjoint pass, input `mode`:
// 0: A = conj(-i k_0 G) v = i k_0 G v;  1: A += G v (the input is i (k_1 P_1 + k_2 P_2))
template <typename T, int LD>
struct AccDst {
  cx_t<T>* p;
  GreenSeq<T> gs;
  int mode;
  __device__ __forceinline__ void st(int row, int c, cx_t<T> v) const {
    using C = cx_t<T>;
    const int f0 = freq_of(row, gs.n);
    const T g = gs.g(f0);
    C* q = p + srow(row) * LD + c;
    if (mode == 1) {
      *q = cadd(*q, cmake<C>(v.x * g, v.y * g));
    } else {
      const T s = (T)gs.fc(0, f0) * g;
      *q = cmake<C>(-v.y * s, v.x * s);
    }
  }
};

template <typename T, int N>
__device__ __forceinline__ GreenSeq<T> green_seq(const ZSeq& q, const T* coef, const T* dtab) {
  GreenSeq<T> gs;
  gs.coef = coef[q.b];
  gs.n12 = q.f1 * q.f1 + q.f2 * q.f2;
  gs.f1 = q.f1;
  gs.f2 = q.f2;
  gs.dtab = dtab;
  gs.n = N;
  gs.d12 = dtab ? dtab[q.f1 < 0 ? q.f1 + N : q.f1] * dtab[q.f2] : (T)1;
  return gs;
}

// Forward force: delta^ (after x, y) --z FFT--> * (-i k_0 G), * G --z IFFT--> z force, U
template <typename T, int L>
__global__ void __launch_bounds__(FusedTile<T, L>::NT)
k_fused_z_force(ZJob<T> job, int ntiles_main, const cx_t<T>* __restrict__ tw) {
  using C = cx_t<T>;
  using TL = FusedTile<T, L>;
  constexpr int TILE = skew_rows(L) * TL::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* A = reinterpret_cast<C*>(smem_raw);
  C* B = A + TILE;
  const bool side = blockIdx.x >= (unsigned)ntiles_main;
  const int s = (side ? blockIdx.x - ntiles_main : blockIdx.x) * TL::TC + threadIdx.x % TL::TC;
  const int nseq = side ? job.batch * L : job.batch * L * (L / 2);
  ZSeq q = zseq<L>(s, side, job.batch);
  q.valid = q.valid && s < nseq;
  GlobalSeq<C> gin{job.in[0] + q.base, q.es, q.valid};
  SmemTile<C, TL::LD> ta{A}, tb{B};
  fft_tile<T, L, TL::TC, TL::NT, -1>(gin, ta, ta, tw);
  __syncthreads();
  const GreenSeq<T> gs = green_seq<T, L>(q, job.coef, job.dtab);
#pragma unroll 1
  for (int c = 0; c < 2; ++c) {
    MulSrc<T, TL::LD> src{A, gs, c};
    GlobalSeq<C> gout{pick(job.out, c) + q.base, q.es, q.valid};
    fft_tile<T, L, TL::TC, TL::NT, +1>(src, tb, gout, tw);
  }
}

// Adjoint: P_0, V = i (k_1 P_1 + k_2 P_2) (after x, y) --z FFT--> G (i k_0 P_0 + V)
// --z IFFT--> psi
template <typename T, int L>
__global__ void __launch_bounds__(FusedTile<T, L>::NT)
k_fused_z_adjoint(ZJob<T> job, int ntiles_main, const cx_t<T>* __restrict__ tw) {
  using C = cx_t<T>;
  using TL = FusedTile<T, L>;
  constexpr int TILE = skew_rows(L) * TL::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* A = reinterpret_cast<C*>(smem_raw);
  C* B = A + TILE;
  const bool side = blockIdx.x >= (unsigned)ntiles_main;
  const int s = (side ? blockIdx.x - ntiles_main : blockIdx.x) * TL::TC + threadIdx.x % TL::TC;
  const int nseq = side ? job.batch * L : job.batch * L * (L / 2);
  ZSeq q = zseq<L>(s, side, job.batch);
  q.valid = q.valid && s < nseq;
  const GreenSeq<T> gs = green_seq<T, L>(q, job.coef, job.dtab);
  SmemTile<C, TL::LD> ta{A}, tb{B};
#pragma unroll 1
  for (int c = 0; c < 2; ++c) {
    GlobalSeq<C> gin{pick(job.in, c) + q.base, q.es, q.valid};
    AccDst<T, TL::LD> acc{A, gs, c};
    fft_tile<T, L, TL::TC, TL::NT, -1>(gin, tb, acc, tw);
    __syncthreads();
  }
  GlobalSeq<C> gout{job.out[0] + q.base, q.es, q.valid};
  fft_tile<T, L, TL::TC, TL::NT, +1>(ta, tb, gout, tw);
}

// ---------------------------------------------------------------- launchers
template <typename T, int L>
static void set_smem(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) ensure_smem_attr(fn, (int)bytes);
}

template <typename T, int L, int DIR>
static void launch_cols_L(const SeqMap& mm, const SeqMap& ms, const ColBufs<T>& bufs, int nbuf,
                          const cx_t<T>* tw, cudaStream_t st) {
  using TL = ColTile<T, L>;
  const int ntm = (mm.nseq + TL::TC - 1) / TL::TC;
  const int nts = ms.nseq > 0 ? (ms.nseq + TL::TC - 1) / TL::TC : 0;
  const size_t sm = TL::SMEM;
  auto fn = k_fft_cols<T, L, DIR>;
  set_smem<T, L>((const void*)fn, sm);
  dim3 grid(ntm + nts, nbuf);
  fn<<<grid, TL::NT, sm, st>>>(mm, ms, ntm, bufs, tw + L);
}

template <typename T, int L, int MODE>
static void launch_cols_yx_L(const SeqMap& mm, const SeqMap& ms, const ColBufs<T>& bufs, const cx_t<T>* tw,
                             cudaStream_t st) {
  using TL = ColTile<T, L>;
  const int ntm = (mm.nseq + TL::TC - 1) / TL::TC;
  const int nts = ms.nseq > 0 ? (ms.nseq + TL::TC - 1) / TL::TC : 0;
  const size_t sm = 2 * (size_t)TL::SMEM;
  auto fn = k_fft_cols_yx<T, L, MODE>;
  set_smem<T, L>((const void*)fn, sm);
  fn<<<ntm + nts, TL::NT, sm, st>>>(mm, ms, ntm, bufs, tw + L);
}

template <typename T, int L>
static void launch_r2c_L(const RowJob<T>& job, int nbuf, int nrows, const cx_t<T>* tw, cudaStream_t st) {
  using TL = RowTile<T, L>;
  const size_t sm = TL::SMEM;
  dim3 grid(((nrows + TL::TR - 1) / TL::TR) * nbuf, 1);
  auto fn = k_fft_x_r2c<T, L>;
  set_smem<T, L>((const void*)fn, sm);
  fn<<<grid, TL::NT, sm, st>>>(job, nrows, nbuf, tw + L, tw + 2 * L);
}

template <typename T, int L>
static void launch_c2r_L(const RowJob<T>& job, int nbuf, int nrows, const cx_t<T>* tw, cudaStream_t st) {
  using TL = RowTile<T, L>;
  const size_t sm = TL::SMEM;
  dim3 grid((nrows + TL::TR - 1) / TL::TR, nbuf);
  auto fn = k_fft_x_c2r<T, L>;
  set_smem<T, L>((const void*)fn, sm);
  fn<<<grid, TL::NT, sm, st>>>(job, nrows, tw + L, tw + 2 * L);
}

template <typename T, int L>
static void launch_fused_L(const ZJob<T>& job, bool adjoint, const cx_t<T>* tw, cudaStream_t st) {
  using TL = FusedTile<T, L>;
  const int ntm = (job.batch * L * (L / 2) + TL::TC - 1) / TL::TC;
  const int nts = (job.batch * L + TL::TC - 1) / TL::TC;
  const size_t sm = 2 * (size_t)TL::SMEM;
  if (adjoint) {
    auto fn = k_fused_z_adjoint<T, L>;
    set_smem<T, L>((const void*)fn, sm);
    fn<<<ntm + nts, TL::NT, sm, st>>>(job, ntm, tw + L);
  } else {
    auto fn = k_fused_z_force<T, L>;
    set_smem<T, L>((const void*)fn, sm);
    fn<<<ntm + nts, TL::NT, sm, st>>>(job, ntm, tw + L);
  }
}

template <typename T, int L> static int tiles_of() { return L * ((L / 2) / TmaTile<T, L>::TC); }

template <typename T, int L, int DIR, int KIND>
static void launch_tma_L(const CUtensorMap* maps, const CUtensorMap* omaps, const TmaJob<T>& job, int tiles,
                         const cx_t<T>* tw, int nsm, cudaStream_t st) {
  using TT = TmaTile<T, L, typename TmaPlanOf<T, L, KIND>::type>;
  TmaMaps m{}, om{};
  const int nomaps = (KIND == 1 || KIND == 3) ? 2 : ((KIND == 2 || KIND == 4) ? 1 : 0);
  for (int i = 0; i < nomaps; ++i) om.m[i] = omaps[i];
  const int nmaps = KIND == 0 ? job.nbuf : ((KIND == 2 || KIND == 4) ? 2 : 1);
  for (int i = 0; i < nmaps; ++i) m.m[i] = maps[i];
  const size_t sm = KIND == 0 ? 3 * (size_t)TT::BYTES + 1024 : 3 * (size_t)TT::BYTES + (size_t)L * sizeof(cx_t<T>) + 1024;
  auto fn = k_cols_tma<T, L, DIR, KIND>;
  ensure_smem_attr((const void*)fn, (int)sm);
  const int items = KIND == 0 ? job.nbuf * tiles : tiles;
  const int grid = items < nsm ? items : nsm;
  fn<<<grid, TT::NT, sm, st>>>(m, om, job, tiles, tw + L);
}

#define PMGB_DISPATCH_TMA(L_, CALL)                                                 \
  switch (L_) {                                                                     \
    case 128: { constexpr int LL = 128; CALL; } break;                              \
    case 256: { constexpr int LL = 256; CALL; } break;                              \
    case 512: { constexpr int LL = 512; CALL; } break;                              \
    case 1024: { constexpr int LL = 1024; CALL; } break;                            \
    default: return PM_ERR_ARG;                                                     \
  }

template <typename T>
int fft_cols_tma(int n, int batch, int dir, int zaxis, const CUtensorMap* maps, cx_t<T>* const* bufs, int nb,
                 const cx_t<T>* tw, const WaitCtl& wc, int nsm, cudaStream_t st) {
  TmaJob<T> job{};
  job.batch = batch;
  for (int i = 0; i < nb; ++i) job.out[i] = bufs[i];
  job.nbuf = nb;
  job.zaxis = zaxis;
  job.err = wc.err;
  job.first_wait = wc.first_wait;
  if (dir < 0) {
    PMGB_DISPATCH_TMA(n, (launch_tma_L<T, LL, -1, 0>(maps, nullptr, job, batch * tiles_of<T, LL>(), tw, nsm, st)));
  } else {
    PMGB_DISPATCH_TMA(n, (launch_tma_L<T, LL, +1, 0>(maps, nullptr, job, batch * tiles_of<T, LL>(), tw, nsm, st)));
  }
  return PM_OK;
}

template <typename T>
int fft_ysplit_tma(int n, int batch, const CUtensorMap* umaps, cx_t<T>* u, cx_t<T>* out1, const cx_t<T>* tw,
                   const WaitCtl& wc, int nsm, cudaStream_t st) {
  TmaJob<T> job{};
  job.out[0] = u;
  job.out[1] = out1;
  job.nbuf = 1;
  job.zaxis = 0;
  job.batch = batch;
  job.err = wc.err;
  job.first_wait = wc.first_wait;
  PMGB_DISPATCH_TMA(n, (launch_tma_L<T, LL, +1, 3>(umaps, umaps, job, batch * tiles_of<T, LL>(), tw, nsm, st)));
  return PM_OK;
}

template <typename T>
int fft_ymerge_tma(int n, int batch, const CUtensorMap* pmaps, cx_t<T>* p1, const cx_t<T>* tw, const WaitCtl& wc, int nsm,
                   cudaStream_t st) {
  TmaJob<T> job{};
  job.out[0] = p1;
  job.nbuf = 1;
  job.zaxis = 0;
  job.batch = batch;
  job.err = wc.err;
  job.first_wait = wc.first_wait;
  PMGB_DISPATCH_TMA(n, (launch_tma_L<T, LL, -1, 4>(pmaps, &pmaps[0], job, batch * tiles_of<T, LL>(), tw, nsm, st)));
  return PM_OK;
}

template <typename T>
int fft_fused_tma(int n, bool adjoint, const CUtensorMap* maps, const CUtensorMap* omaps, const ZJob<T>& zj,
                  const cx_t<T>* tw, const WaitCtl& wc, int nsm, cudaStream_t st) {
  TmaJob<T> job{};
  for (int i = 0; i < 3; ++i) job.out[i] = zj.out[i];
  job.nbuf = 1;
  job.zaxis = 1;
  job.batch = zj.batch;
  job.coef = zj.coef;
  job.dtab = zj.dtab;
  job.err = wc.err;
  job.first_wait = wc.first_wait;
  if (adjoint) {
    PMGB_DISPATCH_TMA(n, (launch_tma_L<T, LL, +1, 2>(maps, omaps, job, zj.batch * tiles_of<T, LL>(), tw, nsm, st)));
  } else {
    PMGB_DISPATCH_TMA(n, (launch_tma_L<T, LL, +1, 1>(maps, omaps, job, zj.batch * tiles_of<T, LL>(), tw, nsm, st)));
  }
  return PM_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).  The
// spectrum main array is viewed as a 4-D tensor of int64 words: (kx words, y, z, batch).
template <typename T, int L>
static int make_maps_L(int batch, cx_t<T>* buf, CUtensorMap* ymap, CUtensorMap* zmap) {
  using Fn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                          const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                          CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Fn encode = nullptr;
  if (!encode) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !f)
      return PM_ERR_CUDA;
    encode = (Fn)f;
  }
  using TT = TmaTile<T, L>;
  constexpr int eb = (int)sizeof(cx_t<T>);
  constexpr int ZB = TT::ZB;
  // main array as (kx words, z mod ZB, y, z / ZB, instance): row (z, y) at
  // ((z / ZB) L + y) ZB + z mod ZB (spec_row)
  const cuuint64_t dims[5] = {(cuuint64_t)(L / 2) * TT::W, (cuuint64_t)ZB, (cuuint64_t)L, (cuuint64_t)(L / ZB),
                              (cuuint64_t)batch};
  const cuuint64_t strides[4] = {(cuuint64_t)(L / 2) * eb, (cuuint64_t)ZB * (L / 2) * eb,
                                 (cuuint64_t)L * ZB * (L / 2) * eb, (cuuint64_t)spec_len_cx(L) * eb};
  const cuuint32_t ybox[5] = {(cuuint32_t)(TT::TC * TT::W), 1, (cuuint32_t)TT::RB, 1, 1};
  const cuuint32_t zbox[5] = {(cuuint32_t)(TT::TC * TT::W), (cuuint32_t)ZB, 1, (cuuint32_t)(TT::RB / ZB), 1};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const CUresult r1 = encode(ymap, CU_TENSOR_MAP_DATA_TYPE_INT64, 5, (void*)buf, dims, strides, ybox, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  const CUresult r2 = encode(zmap, CU_TENSOR_MAP_DATA_TYPE_INT64, 5, (void*)buf, dims, strides, zbox, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return (r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS) ? PM_OK : PM_ERR_CUDA;
}

template <typename T>
int make_spec_tensor_maps(int n, int batch, cx_t<T>* buf, CUtensorMap* ymap, CUtensorMap* zmap) {
  PMGB_DISPATCH_TMA(n, return (make_maps_L<T, LL>(batch, buf, ymap, zmap)));
  return PM_ERR_ARG;
}

#define PMGB_DISPATCH_L(L_, CALL)                                                   \
  switch (L_) {                                                                     \
    case 2: { constexpr int LL = 2; CALL; } break;                                  \
    case 4: { constexpr int LL = 4; CALL; } break;                                  \
    case 8: { constexpr int LL = 8; CALL; } break;                                  \
    case 16: { constexpr int LL = 16; CALL; } break;                                \
    case 32: { constexpr int LL = 32; CALL; } break;                                \
    case 64: { constexpr int LL = 64; CALL; } break;                                \
    case 128: { constexpr int LL = 128; CALL; } break;                              \
    case 256: { constexpr int LL = 256; CALL; } break;                              \
    case 512: { constexpr int LL = 512; CALL; } break;                              \
    case 1024: { constexpr int LL = 1024; CALL; } break;                            \
    default: return PM_ERR_ARG;                                                     \
  }

template <typename T>
int fft_cols(int n, int dir, const SeqMap& mm, const SeqMap& ms, const ColBufs<T>& bufs, int nbuf,
             const cx_t<T>* tw, cudaStream_t st) {
  if (dir < 0) {
    PMGB_DISPATCH_L(n, (launch_cols_L<T, LL, -1>(mm, ms, bufs, nbuf, tw, st)));
  } else {
    PMGB_DISPATCH_L(n, (launch_cols_L<T, LL, +1>(mm, ms, bufs, nbuf, tw, st)));
  }
  return PM_OK;
}

template <typename T>
int fft_cols_split(int n, const SeqMap& mm, const SeqMap& ms, cx_t<T>* u, cx_t<T>* out1, const cx_t<T>* tw,
                   cudaStream_t st) {
  ColBufs<T> b{};
  b.p[0] = u;
  b.p[1] = out1;
  PMGB_DISPATCH_L(n, (launch_cols_yx_L<T, LL, 1>(mm, ms, b, tw, st)));
  return PM_OK;
}

template <typename T>
int fft_cols_merge(int n, const SeqMap& mm, const SeqMap& ms, cx_t<T>* p1, cx_t<T>* p2, const cx_t<T>* tw,
                   cudaStream_t st) {
  ColBufs<T> b{};
  b.p[0] = p1;
  b.p[1] = p2;
  PMGB_DISPATCH_L(n, (launch_cols_yx_L<T, LL, 2>(mm, ms, b, tw, st)));
  return PM_OK;
}

template <typename T>
int fft_x_r2c(int n, const RowJob<T>& job, int nbuf, int nrows, const cx_t<T>* tw,
              cudaStream_t st) {
  if (n < 4 || n > 1024) return PM_ERR_ARG;
  PMGB_DISPATCH_L(n / 2, (launch_r2c_L<T, (LL < 512 ? LL : 512)>(job, nbuf, nrows, tw, st)));
  return PM_OK;
}

template <typename T, int L, int Q>
static void launch_c2r4_LQ(const RowJob<T>& job, int nrows, int dq, void* out, signed char* fexp, const cx_t<T>* tw,
                           cudaStream_t st) {
  using TL = C2R4Tile<T, L, Q>;
  if constexpr (RowTile<T, L>::TR % 4 == 0 && (TL::TR * L) % TL::P::RMAX == 0) {
    const size_t sm = TL::SMEM;
    auto fn = k_fft_x_c2r4<T, L, Q, false>;
    if constexpr (sizeof(T) == 4)
      if (fexp) fn = k_fft_x_c2r4<T, L, Q, true>;
    set_smem<T, L>((const void*)fn, sm);
    fn<<<(nrows + TL::RT - 1) / TL::RT, TL::NT, sm, st>>>(job, nrows, dq, out, fexp, tw + L, tw + 2 * L);
  }
}
template <typename T, int L>
static void launch_c2r4_L(const RowJob<T>& job, int nrows, int dq, void* out, signed char* fexp, const cx_t<T>* tw,
                          cudaStream_t st) {
  if (job.b[3].spec) launch_c2r4_LQ<T, L, 4>(job, nrows, dq, out, fexp, tw, st);
  else launch_c2r4_LQ<T, L, 3>(job, nrows, dq, out, fexp, tw, st);
}

template <typename T>
int fft_x_c2r4(int n, const RowJob<T>& job, int nrows, int dq, void* out, signed char* fexp, const cx_t<T>* tw,
               cudaStream_t st) {
  if (n < 8 || n > 1024) return PM_ERR_ARG;
  if (fexp && sizeof(T) != 4) return PM_ERR_ARG;
  PMGB_DISPATCH_L(n / 2, (launch_c2r4_L<T, (LL < 512 ? LL : 512)>(job, nrows, dq, out, fexp, tw, st)));
  return PM_OK;
}

template <typename T>
int fft_x_c2r(int n, const RowJob<T>& job, int nbuf, int nrows, const cx_t<T>* tw, cudaStream_t st) {
  if (n < 4 || n > 1024) return PM_ERR_ARG;
  PMGB_DISPATCH_L(n / 2, (launch_c2r_L<T, (LL < 512 ? LL : 512)>(job, nbuf, nrows, tw, st)));
  return PM_OK;
}

template <typename T, int L>
static void launch_fused_side_L(const ZJob<T>& job, bool adjoint, const cx_t<T>* tw, cudaStream_t st) {
  using TL = FusedTile<T, L>;
  const int nts = (job.batch * L + TL::TC - 1) / TL::TC;
  const size_t sm = 2 * (size_t)TL::SMEM;
  if (adjoint) {
    auto fn = k_fused_z_adjoint<T, L>;
    set_smem<T, L>((const void*)fn, sm);
    fn<<<nts, TL::NT, sm, st>>>(job, 0, tw + L);
  } else {
    auto fn = k_fused_z_force<T, L>;
    set_smem<T, L>((const void*)fn, sm);
    fn<<<nts, TL::NT, sm, st>>>(job, 0, tw + L);
  }
}

template <typename T>
int fft_fused_side(int n, const ZJob<T>& job, bool adjoint, const cx_t<T>* tw, cudaStream_t st) {
  if (n < 4) return PM_ERR_ARG;
  PMGB_DISPATCH_L(n, (launch_fused_side_L<T, (LL < 4 ? 4 : LL)>(job, adjoint, tw, st)));
  return PM_OK;
}

template <typename T>
int fft_fused_z(int n, const ZJob<T>& job, bool adjoint, const cx_t<T>* tw, cudaStream_t st) {
  if (n < 4) return PM_ERR_ARG;
  PMGB_DISPATCH_L(n, (launch_fused_L<T, (LL < 4 ? 4 : LL)>(job, adjoint, tw, st)));
  return PM_OK;
}

}  // namespace pmgb
