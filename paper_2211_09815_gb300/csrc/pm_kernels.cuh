// Particle and mesh kernels of the PM hot path (besides the FFT passes), templated on the
// real type.  Included once per precision.
//
//  k_scatter        CIC mass (and adjoint pi) assignment, Sec. 2.2 Eq. 10, int64 fixed point
//                   with global atomics (the allocation-free density entry point; the
//                   engine assigns by mesh tiles, bin_kernels.cuh)
//  k_gather_fwd     CIC force gather + kick / kick / drift of Eq. 16 (one launch per step);
//                   counts the deposit bins of the new positions for the next step
//  k_gather_adj     CIC gather of a and alpha (Eq. 49 F line) + reverse kicks and drift of
//                   Eq. 49, FP64 partials of the theta terms of Eq. 51; bin counts as above
//  k_adjoint_init   xi_n = dJ/dx_n (density cotangent through the CIC weight gradient), pi_n
//  k_obs_cotangent  the same cotangent of an observed intermediate state, added to xi_j
//  k_density_out, k_mse, k_za_mul, k_za_adj_mul, k_ic_state, k_ic_adj_prep, k_final_theta,
//  k_lpt_hess, k_lpt_source, k_lpt_source_adj, k_lpt_hess_adj, k_ic_state2
#pragma once
#include <cuda_fp16.h>
#include "common.cuh"
#include "pm_internal.h"

namespace pmgb {

constexpr int kPtclThreads = 256;
constexpr int kMaxRedBlocks = 1024;

// Lattice and mesh geometry of one instance.
template <typename T> struct Geo {
  int lg_np;      // log2 n_ptcl
  int np, nm;     // particles / mesh nodes per side
  int ratio;      // nm / np
  T inv_l;        // 1 / cell size
  long long N;    // particles per instance
  long long M;    // mesh cells per instance
};

// correctly rounded products and fused multiply-adds, never re-associated or contracted
// differently by the compiler: the forward and reverse passes gather the same force on a
// particle bit for bit
template <typename T> __device__ __forceinline__ T mul_rn(T a, T b);
template <> __device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }
template <> __device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }
template <typename T> __device__ __forceinline__ T fma_rn(T a, T b, T c);
template <> __device__ __forceinline__ float fma_rn<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ double fma_rn<double>(double a, double b, double c) { return __fma_rn(a, b, c); }


// Cell index and fraction along each axis for particle i at displacement s (floor
// convention: u = q/l + s/l with q/l = j*ratio + 1/2; the integer part of q/l is added
// separately so that the fraction keeps the precision of s, not of x).
template <typename T>
__device__ __forceinline__ void cic_cell(const Geo<T>& g, long long i, const T s[3], int cell[3], T t[3]) {
  const int j[3] = {(int)(i >> (2 * g.lg_np)), (int)((i >> g.lg_np) & (g.np - 1)), (int)(i & (g.np - 1))};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T v = fma_rn<T>(s[c], g.inv_l, (T)0.5);
    const T f = floor(v);
    t[c] = v - f;
    cell[c] = (j[c] * g.ratio + (int)f) & (g.nm - 1);
  }
}

// Work index -> lattice particle index: 8^3 Lagrangian blocks (x fastest inside a block,
// so a warp reads 8 x 4 particles in full 32-byte segments) visited in Morton order of the
// block coordinates, so that the particles in flight at any moment -- and the mesh cells
// they scatter to or gather from -- form a compact region that stays in L2.
__device__ __forceinline__ unsigned long long morton_compact3(unsigned long long x) {
  x &= 0x1249249249249249ull;
  x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
  x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
  x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
  x = (x ^ (x >> 32)) & 0x1fffffull;
  return x;
}
template <typename T>
__device__ __forceinline__ long long particle_of(const Geo<T>& g, long long w) {
  const int tb = g.lg_np < 3 ? g.lg_np : 3;                 // block side 2^tb
  const long long inner = w & ((1LL << (3 * tb)) - 1);
  const unsigned long long blk = (unsigned long long)(w >> (3 * tb));
  const int mask = (1 << tb) - 1;
  const long long x = ((long long)morton_compact3(blk) << tb) | (inner & mask);
  const long long y = ((long long)morton_compact3(blk >> 1) << tb) | ((inner >> tb) & mask);
  const long long z = ((long long)morton_compact3(blk >> 2) << tb) | (inner >> (2 * tb));
  return (z << (2 * g.lg_np)) | (y << g.lg_np) | x;
}

template <typename T>
__device__ __forceinline__ long long corner_index(const Geo<T>& g, const int cell[3], int d) {
  const int m = g.nm - 1;
  const int i0 = (cell[0] + ((d >> 2) & 1)) & m;
  const int i1 = (cell[1] + ((d >> 1) & 1)) & m;
  const int i2 = (cell[2] + (d & 1)) & m;
  return ((long long)i0 * g.nm + i1) * g.nm + i2;
}

// The eight CIC corners of the [cell][4] force mesh: FP32 V4 per cell, or (H, FP32 path
// only) the FP16 mesh of k_fft_x_c2r4<..., true>: four halves per cell, each field of a row
// (fixed z, y) scaled by 2^-e with e an int8 of the row's packed quadruple in fexp.
template <typename T, bool H>
__device__ __forceinline__ void load_corners(const Geo<T>& g, const void* __restrict__ fvec,
                                             const int* __restrict__ fexp, int b, const int cell[3], V4<T> fv[8]) {
  if constexpr (!H) {
    const V4<T>* F = reinterpret_cast<const V4<T>*>(fvec) + (long long)b * g.M;
#pragma unroll
    for (int d = 0; d < 8; ++d) fv[d] = F[corner_index(g, cell, d)];
  } else {
    static_assert(sizeof(T) == 4, "the FP16 force mesh is an FP32-path form");
    const uint2* F = reinterpret_cast<const uint2*>(fvec) + (long long)b * g.M;
    const int* E = fexp + (long long)b * g.nm * g.nm;
    const int m = g.nm - 1;
    int ew[4];   // exponent quadruples of the rows (z0 + dz, y0 + dy), index 2 dz + dy
#pragma unroll
    for (int k = 0; k < 4; ++k) ew[k] = __ldg(E + ((cell[0] + (k >> 1)) & m) * g.nm + ((cell[1] + (k & 1)) & m));
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const uint2 u = __ldg(F + corner_index(g, cell, d));
      const int w = ew[(d >> 1) & 3];
      const float2 lo = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
      const float2 hi = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
      fv[d] = V4<T>{lo.x * __int_as_float(((int)(signed char)(w & 0xFF) + 127) << 23),
                    lo.y * __int_as_float(((int)(signed char)((w >> 8) & 0xFF) + 127) << 23),
                    hi.x * __int_as_float(((int)(signed char)((w >> 16) & 0xFF) + 127) << 23),
                    hi.y * __int_as_float(((int)(signed char)((w >> 24) & 0xFF) + 127) << 23)};
    }
  }
}

template <typename T> __device__ __forceinline__ long long to_fixed(T v);
template <> __device__ __forceinline__ long long to_fixed<float>(float v) { return f2ll_rn(v); }
template <> __device__ __forceinline__ long long to_fixed<double>(double v) { return __double2ll_rn(v); }

// Exactly reversible particle state (pm_config.fixed_state): displacement and momentum held
// as 64-bit integers, U = s / l in units of 2^-kFixES cells and W = p / l in units of
// 2^-kFixEP cells per unit of drift factor.  A kick adds round(a K / l 2^kFixEP), a drift
// round(w D 2^kFixES) with w the working-precision value of W; the reverse pass subtracts
// the same rounded increments (the same forces at the same positions), so it recovers the
// forward states bit for bit.  The kernels that read positions and momenta see working-
// precision shadows s = U l 2^-kFixES, p = W l 2^-kFixEP.
constexpr int kFixES = 40, kFixEP = 36;
template <typename T> struct FixState {
  long long* u;   // [batch][3][N] or null: floating-point state
  long long* w;
  T to_w;         // 2^kFixEP / l: momentum increment -> W units
  T from_u;       // l 2^-kFixES: U -> displacement
  T from_w;       // l 2^-kFixEP: W -> momentum
  T w_cells;      // 2^-kFixEP: W -> cells per unit of drift factor
  T du;           // 2^kFixES: cells -> U units
};
template <typename T> __device__ __forceinline__ T fix_to_real(long long v);
template <> __device__ __forceinline__ float fix_to_real<float>(long long v) { return ll2f_rn(v); }
template <> __device__ __forceinline__ double fix_to_real<double>(long long v) { return (double)v; }

// Deterministic block sum of one double per thread (fixed shuffle tree + fixed warp order).
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  return r;
}

__device__ __forceinline__ float block_max(float v, float* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  float r = 0.f;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r = fmaxf(r, sh[i]);
  return r;
}

// Per-thread partial sums of the theta terms: compensated (Kahan) summation in the working
// precision, handed to the FP64 block reduction; FP64 arithmetic is slow on this part.
template <typename T> struct KahanAcc {
  T s = 0, c = 0;
  __device__ __forceinline__ void add(T v) {
    const T y = v - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <typename T> __device__ __forceinline__ float abs_up(T v);
template <> __device__ __forceinline__ float abs_up<float>(float v) { return fabsf(v); }
template <> __device__ __forceinline__ float abs_up<double>(double v) { return __double2float_ru(fabs(v)); }

// ------------------------------------------------------------------------- scatter
// NQ = 1: acc[cell] += W * 2^e_d (weights).  NQ = 4: acc is [cell][4] and receives the
// weight and pi_c * W * 2^e_c (c = 0..2) in one 32-byte sector per cell.
template <typename T, int NQ>
__global__ void __launch_bounds__(kPtclThreads)
k_scatter(Geo<T> g, const T* __restrict__ s, const T* __restrict__ pi, unsigned long long* acc, int e_d,
          const int* __restrict__ e_pi) {
  const int b = blockIdx.y;
  const T* sb = s + (long long)b * 3 * g.N;
  const long long mo = (long long)b * g.M;
  const T sd = (T)ldexp(1.0, e_d);
  T sp[3] = {0, 0, 0};
  const T* pb = nullptr;
  if constexpr (NQ == 4) {
    pb = pi + (long long)b * 3 * g.N;
#pragma unroll
    for (int c = 0; c < 3; ++c) sp[c] = (T)ldexp(1.0, e_pi[c * gridDim.y + b]);
  }
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < g.N;
       w += (long long)gridDim.x * blockDim.x) {
    const long long i = particle_of(g, w);
    const T sv[3] = {sb[i], sb[g.N + i], sb[2 * g.N + i]};
    int cell[3];
    T t[3];
    cic_cell(g, i, sv, cell, t);
    T pv[3] = {0, 0, 0};
    if constexpr (NQ == 4) {
      pv[0] = pb[i] * sp[0];
      pv[1] = pb[g.N + i] * sp[1];
      pv[2] = pb[2 * g.N + i] * sp[2];
    }
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const T w = ((d & 4) ? t[0] : (T)1 - t[0]) * ((d & 2) ? t[1] : (T)1 - t[1]) * ((d & 1) ? t[2] : (T)1 - t[2]);
      const long long idx = mo + corner_index(g, cell, d);
      if constexpr (NQ == 1) {
        atomicAdd(acc + idx, (unsigned long long)to_fixed<T>(w * sd));
      } else {
        unsigned long long* q = acc + 4 * idx;
        atomicAdd(q, (unsigned long long)to_fixed<T>(w * sd));
        atomicAdd(q + 1, (unsigned long long)to_fixed<T>(pv[0] * w));
        atomicAdd(q + 2, (unsigned long long)to_fixed<T>(pv[1] * w));
        atomicAdd(q + 3, (unsigned long long)to_fixed<T>(pv[2] * w));
      }
    }
  }
}

// fixed-point exponents of the pi scatters from max|pi_c| (layout [c][batch]): one
// contribution |pi| W 2^e is below 2^(E + e) and the sum over one cell below N 2^(E + e),
// with max|pi| < 2^E; e = top - E keeps them below 2^top and 2^(lg N + top) (top: see
// fixed_top).
static __global__ void k_pi_exponents(const unsigned* __restrict__ pimax, int* __restrict__ e_pi, int nq, int top) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  const float mx = __uint_as_float(pimax[i]);
  int e = 0;
  if (mx > 0.f && isfinite(mx)) {
    const int E = ilogbf(mx) + 1;   // mx < 2^E
    e = top - E;
    if (e > 100) e = 100;
  }
  e_pi[i] = e;
}

// Bits of one fixed-point contribution of the assignment.  FP32: 2^30, so that a
// contribution is an int32 (its 24-bit significand loses nothing there) and the sum over a
// cell of N contributions stays below 2^61 for N <= 2^31; FP64: 61 - lg N, the widest
// quantum the int64 cell sums allow.
template <typename T> inline int fixed_top(int lgN);
template <> inline int fixed_top<float>(int lgN) { return 61 - lgN < 30 ? 61 - lgN : 30; }
template <> inline int fixed_top<double>(int lgN) { return 61 - lgN; }

// A fixed-point contribution as the two 32-bit words of an int64, correctly rounded
// (nearest-even).  FP32 contributions are at most 2^30 in magnitude (fixed_top), so one
// hardware conversion to int32 rounds them (ties to even, symmetric in the sign) and the
// high word is the sign extension.
template <typename T> __device__ __forceinline__ void fixed_words(T v, unsigned& lo, unsigned& hi);
template <> __device__ __forceinline__ void fixed_words<float>(float v, unsigned& lo, unsigned& hi) {
  const int r = __float2int_rn(v);
  lo = (unsigned)r;
  hi = (unsigned)(r >> 31);
}
template <> __device__ __forceinline__ void fixed_words<double>(double v, unsigned& lo, unsigned& hi) {
  const unsigned long long r = (unsigned long long)__double2ll_rn(v);
  lo = (unsigned)r;
  hi = (unsigned)(r >> 32);
}

// ------------------------------------------------------------------ deposit bins
// Bins of the tile-owner deposit (bin_kernels.cuh): mesh tiles of 2^lx x 2^ly x 2^lz cells
// (x = array axis 2), and per tile a class of three bits, set when the particle's cell is on
// the tile's last layer along x, y or z (its CIC cloud reaches into the next tile there).
struct BinGeo {
  int lx, ly, lz;       // log2 of the tile extent along axes 2, 1, 0
  int ntx, nty, ntz;    // tiles per axis
  int ntiles;           // per instance
  long long nkeys;      // bins per instance = 8 ntiles
};

inline BinGeo make_bin_geo(int lg_nm, int lx, int ly, int lz) {
  BinGeo b;
  b.lx = lx < lg_nm ? lx : lg_nm;
  b.ly = ly < lg_nm ? ly : lg_nm;
  b.lz = lz < lg_nm ? lz : lg_nm;
  b.ntx = 1 << (lg_nm - b.lx);
  b.nty = 1 << (lg_nm - b.ly);
  b.ntz = 1 << (lg_nm - b.lz);
  b.ntiles = b.ntx * b.nty * b.ntz;
  b.nkeys = 8LL * b.ntiles;
  return b;
}

// class bits of a cell: on the last layer of its tile along x (bit 0), y (bit 1), z (bit 2)
__device__ __forceinline__ unsigned bin_class(const BinGeo& bg, const int c[3]) {
  const unsigned mx = (1u << bg.lx) - 1, my = (1u << bg.ly) - 1, mz = (1u << bg.lz) - 1;
  return (unsigned)(((unsigned)c[2] & mx) == mx) | ((unsigned)(((unsigned)c[1] & my) == my) << 1) |
         ((unsigned)(((unsigned)c[0] & mz) == mz) << 2);
}
__device__ __forceinline__ unsigned bin_key(const BinGeo& bg, const int c[3]) {
  const unsigned tile = (((unsigned)c[0] >> bg.lz) * bg.nty + ((unsigned)c[1] >> bg.ly)) * bg.ntx + ((unsigned)c[2] >> bg.lx);
  return tile * 8u + bin_class(bg, c);
}

// Count a particle's bin for the next deposit (its key, and a warp-aggregated increment of
// the bin count).  Every lane of the warp calls this together.
template <typename T>
__device__ __forceinline__ void count_bin(const Geo<T>& g, const BinGeo& bg, long long i, const T sv[3], int b,
                                          unsigned* __restrict__ count, unsigned* __restrict__ keys) {
  int cell[3];
  T t[3];
  cic_cell(g, i, sv, cell, t);
  const unsigned key = bin_key(bg, cell);
  keys[(long long)b * g.N + i] = key;
  const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
  if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(count + (long long)b * bg.nkeys + key, (unsigned)__popc(peers));
}

// ---------------------------------------------------------------------- gathers
template <typename T>
struct StepCoef {  // per-instance coefficient tables [batch][n+1], indexed at step j
  const T* kA;
  const T* kB;
  const T* dr;
};

// a = sum_g W f(g);  p += a kA;  (store p_j);  p += a kB;  (store s_j);  s += p dr
template <typename T, bool H = false>
__global__ void __launch_bounds__(kPtclThreads)
k_gather_fwd(Geo<T> g, T* __restrict__ s, T* __restrict__ p, T* __restrict__ a_out,
             const void* __restrict__ fvec, const int* __restrict__ fexp, StepCoef<T> sc, int j, int nstep1,
             T* __restrict__ ck_s,
             T* __restrict__ ck_p, BinGeo bg, unsigned* __restrict__ bcount, unsigned* __restrict__ bkeys,
             T* __restrict__ snap_p = nullptr, FixState<T> fx = FixState<T>{}) {
  const int b = blockIdx.y;
  const T kA = sc.kA[b * nstep1 + j], kB = sc.kB[b * nstep1 + j], dr = sc.dr[b * nstep1 + j];
  T* sb = s + (long long)b * 3 * g.N;
  T* pb = p + (long long)b * 3 * g.N;
  // the displacement of the thread's next particle is read one iteration ahead, so that
  // its latency overlaps this particle's corner loads (each particle has one thread: the
  // value is not written before it is used)
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  T sn[3] = {0, 0, 0};
  if (w < g.N) {
    const long long i0 = particle_of(g, w);
    sn[0] = sb[i0], sn[1] = sb[g.N + i0], sn[2] = sb[2 * g.N + i0];
  }
  for (; w < g.N; w += stride) {
    const long long i = particle_of(g, w);
    T sv[3] = {sn[0], sn[1], sn[2]};
    T pv[3] = {pb[i], pb[g.N + i], pb[2 * g.N + i]};   // in flight with the corner loads
    int cell[3];
    T t[3];
    cic_cell(g, i, sv, cell, t);
    V4<T> fv[8];
    load_corners<T, H>(g, fvec, fexp, b, cell, fv);
    if (w + stride < g.N) {
      const long long in = particle_of(g, w + stride);
      sn[0] = sb[in], sn[1] = sb[g.N + in], sn[2] = sb[2 * g.N + in];
    }
    T a[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const T w0 = (d & 4) ? t[0] : (T)1 - t[0];
      const T w1 = (d & 2) ? t[1] : (T)1 - t[1];
      const T w2 = (d & 1) ? t[2] : (T)1 - t[2];
      const T w = mul_rn<T>(mul_rn<T>(w0, w1), w2);
      a[0] = fma_rn<T>(w, fv[d].x, a[0]);
      a[1] = fma_rn<T>(w, fv[d].y, a[1]);
      a[2] = fma_rn<T>(w, fv[d].z, a[2]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long o = (long long)b * 3 * g.N + c * g.N + i;
      if (fx.u) {
        // fixed-point state: exact integer kicks and drift, shadows for the other kernels
        long long W = fx.w[o], U = fx.u[o];
        W += to_fixed<T>(mul_rn<T>(mul_rn<T>(a[c], kA), fx.to_w));
        if (ck_p || snap_p) pv[c] = mul_rn<T>(fix_to_real<T>(W), fx.from_w);
        if (ck_p) ck_p[o] = pv[c];
        if (snap_p) snap_p[o] = pv[c];
        W += to_fixed<T>(mul_rn<T>(mul_rn<T>(a[c], kB), fx.to_w));
        if (ck_s) ck_s[o] = sv[c];
        U += to_fixed<T>(mul_rn<T>(mul_rn<T>(mul_rn<T>(fix_to_real<T>(W), fx.w_cells), dr), fx.du));
        fx.w[o] = W;
        fx.u[o] = U;
        pv[c] = mul_rn<T>(fix_to_real<T>(W), fx.from_w);
        sv[c] = mul_rn<T>(fix_to_real<T>(U), fx.from_u);
      } else {
        pv[c] += a[c] * kA;
        if (ck_p) ck_p[o] = pv[c];
        if (snap_p) snap_p[o] = pv[c];   // p_j of an observed state
        pv[c] += a[c] * kB;
        if (ck_s) ck_s[o] = sv[c];
        sv[c] += pv[c] * dr;
      }
      pb[c * g.N + i] = pv[c];
      sb[c * g.N + i] = sv[c];
      if (a_out) a_out[o] = a[c];
    }
    // bin of the new position for the next step's deposit (the loop is warp-uniform: N is
    // a multiple of 32 and so is the grid stride)
    if (bcount) count_bin(g, bg, i, sv, b, bcount, bkeys);
  }
}

// Reverse step at force step j (Eq. 49): a_j = sum W f, alpha_j = sum grad W [pi.f + m psi];
// p -= a K1_{j+1}; xi += alpha K1_{j+1}; (p := stored p_j); p -= a K2_j; xi += alpha K2_j;
// s -= p D_j; pi += xi D_j; (s := stored s_{j-1}).  FP64 partials of pi.a and xi.p.
template <typename T, bool H = false>
__global__ void __launch_bounds__(kPtclThreads)
k_gather_adj(Geo<T> g, T mass, T* __restrict__ s, T* __restrict__ p, T* __restrict__ xi, T* __restrict__ pi,
             T* __restrict__ a_out, T* __restrict__ alpha_out, const void* __restrict__ fvec,
             const int* __restrict__ fexp, StepCoef<T> sc, int j, int nstep1,
             const T* __restrict__ ck_p, const T* __restrict__ ck_s, double* __restrict__ part_pa,
             double* __restrict__ part_xp, unsigned* __restrict__ pimax, BinGeo bg, unsigned* __restrict__ bcount,
             unsigned* __restrict__ bkeys, FixState<T> fx = FixState<T>{}) {
  __shared__ double shd[kPtclThreads / 32];
  __shared__ float shf[kPtclThreads / 32];
  const int b = blockIdx.y;
  const T cA = sc.kA[b * nstep1 + j], cB = sc.kB[b * nstep1 + j], dr = sc.dr[b * nstep1 + j];
  const long long po = (long long)b * 3 * g.N;
  const T il = g.inv_l;
  KahanAcc<T> acc_pa, acc_xp;
  float mx[3] = {0.f, 0.f, 0.f};
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < g.N;
       w += (long long)gridDim.x * blockDim.x) {
    const long long i = particle_of(g, w);
    T sv[3], pv[3], xv[3], qv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      sv[c] = s[po + c * g.N + i];
      pv[c] = p[po + c * g.N + i];
      xv[c] = xi[po + c * g.N + i];
      qv[c] = pi[po + c * g.N + i];
    }
    int cell[3];
    T t[3];
    cic_cell(g, i, sv, cell, t);
    V4<T> fv[8];
    load_corners<T, H>(g, fvec, fexp, b, cell, fv);
    T a[3] = {0, 0, 0}, al[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const T w0 = (d & 4) ? t[0] : (T)1 - t[0];
      const T w1 = (d & 2) ? t[1] : (T)1 - t[1];
      const T w2 = (d & 1) ? t[2] : (T)1 - t[2];
      const T g0 = (d & 4) ? il : -il, g1 = (d & 2) ? il : -il, g2 = (d & 1) ? il : -il;
      const T h = qv[0] * fv[d].x + qv[1] * fv[d].y + qv[2] * fv[d].z + mass * fv[d].w;
      const T w = mul_rn<T>(mul_rn<T>(w0, w1), w2);
      a[0] = fma_rn<T>(w, fv[d].x, a[0]);
      a[1] = fma_rn<T>(w, fv[d].y, a[1]);
      a[2] = fma_rn<T>(w, fv[d].z, a[2]);
      al[0] += g0 * w1 * w2 * h;
      al[1] += w0 * g1 * w2 * h;
      al[2] += w0 * w1 * g2 * h;
    }
    acc_pa.add(qv[0] * a[0] + qv[1] * a[1] + qv[2] * a[2]);
    long long W[3] = {0, 0, 0};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (fx.u) {
        // the forward's rounded increments, subtracted in reverse order (checkpoints are
        // never combined with the fixed-point state)
        W[c] = fx.w[po + c * g.N + i];
        W[c] -= to_fixed<T>(mul_rn<T>(mul_rn<T>(a[c], cA), fx.to_w));
        W[c] -= to_fixed<T>(mul_rn<T>(mul_rn<T>(a[c], cB), fx.to_w));
        pv[c] = mul_rn<T>(fix_to_real<T>(W[c]), fx.from_w);
      } else {
        pv[c] -= a[c] * cA;
        if (ck_p) pv[c] = ck_p[po + c * g.N + i];
        pv[c] -= a[c] * cB;
      }
      xv[c] += al[c] * cA;
      xv[c] += al[c] * cB;
    }
    acc_xp.add(xv[0] * pv[0] + xv[1] * pv[1] + xv[2] * pv[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (fx.u) {
        long long U = fx.u[po + c * g.N + i];
        U -= to_fixed<T>(mul_rn<T>(mul_rn<T>(mul_rn<T>(fix_to_real<T>(W[c]), fx.w_cells), dr), fx.du));
        fx.u[po + c * g.N + i] = U;
        fx.w[po + c * g.N + i] = W[c];
        sv[c] = mul_rn<T>(fix_to_real<T>(U), fx.from_u);
      } else {
        sv[c] -= pv[c] * dr;
      }
      qv[c] += xv[c] * dr;
      if (ck_s) sv[c] = ck_s[po + c * g.N + i];
      s[po + c * g.N + i] = sv[c];
      p[po + c * g.N + i] = pv[c];
      xi[po + c * g.N + i] = xv[c];
      pi[po + c * g.N + i] = qv[c];
      mx[c] = fmaxf(mx[c], abs_up<T>(qv[c]));
      if (a_out) a_out[po + c * g.N + i] = a[c];
      if (alpha_out) alpha_out[po + c * g.N + i] = al[c];
    }
    if (bcount) count_bin(g, bg, i, sv, b, bcount, bkeys);   // bin for the previous step's deposit
  }
  const double spa = block_sum(acc_pa.value(), shd);
  const double sxp = block_sum(acc_xp.value(), shd);
  if (threadIdx.x == 0 && part_pa) {
    part_pa[(long long)b * gridDim.x + blockIdx.x] = spa;
    part_xp[(long long)b * gridDim.x + blockIdx.x] = sxp;
  }
  if (pimax) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float m = block_max(mx[c], shf);
      if (threadIdx.x == 0) atomicMax(pimax + c * gridDim.y + b, __float_as_uint(m));
    }
  }
}

// xv += m sum_g grad_x W(g - x_i) D(g) over the 8 CIC corners of particle i at
// displacement sv: a density cotangent D carried to the particle position through the
// weight gradient (floor convention, -1/l and +1/l per axis).
template <typename T>
__device__ __forceinline__ void cic_grad_gather(const Geo<T>& g, long long i, const T sv[3], const T* D, T mass,
                                                T xv[3]) {
  const T il = g.inv_l;
  int cell[3];
  T t[3];
  cic_cell(g, i, sv, cell, t);
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    const T w0 = (d & 4) ? t[0] : (T)1 - t[0];
    const T w1 = (d & 2) ? t[1] : (T)1 - t[1];
    const T w2 = (d & 1) ? t[2] : (T)1 - t[2];
    const T g0 = (d & 4) ? il : -il, g1 = (d & 2) ? il : -il, g2 = (d & 1) ? il : -il;
    const T h = mass * __ldg(D + corner_index(g, cell, d));
    xv[0] += g0 * w1 * w2 * h;
    xv[1] += w0 * g1 * w2 * h;
    xv[2] += w0 * w1 * g2 * h;
  }
}

// xi = m sum_g grad W(g - x) dJ/ddelta(g) (+ dJ/dx);  pi = dJ/dp (or 0)
template <typename T>
__global__ void __launch_bounds__(kPtclThreads)
k_adjoint_init(Geo<T> g, T mass, const T* __restrict__ s, const T* __restrict__ djdd, const T* __restrict__ djdx,
               const T* __restrict__ djdp, T* __restrict__ xi, T* __restrict__ pi, unsigned* __restrict__ pimax) {
  __shared__ float shf[kPtclThreads / 32];
  const int b = blockIdx.y;
  const long long po = (long long)b * 3 * g.N;
  float mx[3] = {0.f, 0.f, 0.f};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
       i += (long long)gridDim.x * blockDim.x) {
    T xv[3] = {0, 0, 0};
    if (djdd) {
      const T sv[3] = {s[po + i], s[po + g.N + i], s[po + 2 * g.N + i]};
      cic_grad_gather(g, i, sv, djdd + (long long)b * g.M, mass, xv);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (djdx) xv[c] += djdx[po + c * g.N + i];
      xi[po + c * g.N + i] = xv[c];
      const T q = djdp ? djdp[po + c * g.N + i] : (T)0;
      pi[po + c * g.N + i] = q;
      mx[c] = fmaxf(mx[c], abs_up<T>(q));
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float m = block_max(mx[c], shf);
    if (threadIdx.x == 0) atomicMax(pimax + c * gridDim.y + b, __float_as_uint(m));
  }
}

// Cotangent of an observed intermediate state (Sec. 2.4, objectives on z_0..z_n), added
// when the reverse pass holds its positions x_j:  xi += m sum_g grad W dJ/d delta_j(g)
// + dJ/dx_j.  xi enters nothing before the reverse drift of step j, so the sum is exact
// whatever the kicks between add.
template <typename T>
__global__ void __launch_bounds__(kPtclThreads)
k_obs_cotangent(Geo<T> g, T mass, const T* __restrict__ s, const T* __restrict__ djdd, const T* __restrict__ djdx,
                T* __restrict__ xi) {
  const int b = blockIdx.y;
  const long long po = (long long)b * 3 * g.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
       i += (long long)gridDim.x * blockDim.x) {
    T xv[3] = {0, 0, 0};
    if (djdd) {
      const T sv[3] = {s[po + i], s[po + g.N + i], s[po + 2 * g.N + i]};
      cic_grad_gather(g, i, sv, djdd + (long long)b * g.M, mass, xv);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (djdx) xv[c] += djdx[po + c * g.N + i];
      xi[po + c * g.N + i] += xv[c];
    }
  }
}

// Cotangent v = dJ/dp_j of an observed momentum (Sec. 2.4), added to pi in two parts
// around the reverse step at force step j: the reverse kick K1_{j+1} uses pi, the
// reverse kick K2_j (the one that made p_j) pi + v.  The force VJP is linear in pi, so one
// VJP of pi + c v with c = K2_j / (K1_{j+1} + K2_j) gives both kicks' alpha terms:
//   mode 0 (before the force chain): pi += c v
//   mode 1 (after the reverse step):  pi += (1 - c) v, and the FP64 block sums of v . a_j
//   (the theta term of the K2_j kick that pi + c v does not carry).
// The fixed-point exponent of the next pi deposit is kept valid: max |pi| is folded into
// pimax.
template <typename T>
__global__ void __launch_bounds__(kPtclThreads)
k_obs_momentum(Geo<T> g, T* __restrict__ pi, const T* __restrict__ v, const T* __restrict__ ctab, int j, int nstep1,
               int mode, const T* __restrict__ a, double* __restrict__ part, unsigned* __restrict__ pimax) {
  __shared__ double shd[kPtclThreads / 32];
  __shared__ float shf[kPtclThreads / 32];
  const int b = blockIdx.y;
  const long long po = (long long)b * 3 * g.N;
  const T c = ctab[b * nstep1 + j];
  const T w = mode == 0 ? c : (T)1 - c;
  double acc = 0.0;
  float mx[3] = {0.f, 0.f, 0.f};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x) {
    T va = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const long long o = po + k * g.N + i;
      const T q = pi[o] + w * v[o];
      pi[o] = q;
      mx[k] = fmaxf(mx[k], abs_up<T>(q));
      if (mode == 1) va += v[o] * a[o];
    }
    acc += (double)va;
  }
  if (mode == 1) {
    const double r = block_sum(acc, shd);
    if (threadIdx.x == 0) part[(long long)b * gridDim.x + blockIdx.x] = r;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float m = block_max(mx[k], shf);
    if (threadIdx.x == 0) atomicMax(pimax + k * gridDim.y + b, __float_as_uint(m));
  }
}

// Cotangent of positions observed at a scale factor a between steps j and j + 1 (Sec. 2.4):
// x(a) = q + s_j + Dp_j(a) p_{j+1/2} with the partial drift factor fac = Dp_j(a), taken
// while the reverse pass holds (s_j, p_{j+1/2}) before the force VJP at x_j:
//   u = m sum_g grad W(g - x(a)) dJ/d delta(a)(g) + dJ/dx(a);  xi += u;  pi += fac u;
// and the FP64 block sums of u . p_{j+1/2} (the theta term of Dp_j).
template <typename T>
__global__ void __launch_bounds__(kPtclThreads)
k_obs_interp(Geo<T> g, T mass, const T* __restrict__ s, const T* __restrict__ p, const T* __restrict__ fac_tab,
             const T* __restrict__ djdd, const T* __restrict__ djdx, T* __restrict__ xi, T* __restrict__ pi,
             double* __restrict__ part, unsigned* __restrict__ pimax) {
  __shared__ double shd[kPtclThreads / 32];
  __shared__ float shf[kPtclThreads / 32];
  const int b = blockIdx.y;
  const long long po = (long long)b * 3 * g.N;
  const T fac = fac_tab[b];
  double acc = 0.0;
  float mx[3] = {0.f, 0.f, 0.f};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x) {
    T u[3] = {0, 0, 0};
    const T pv[3] = {p[po + i], p[po + g.N + i], p[po + 2 * g.N + i]};
    if (djdd) {
      const T sa[3] = {s[po + i] + fac * pv[0], s[po + g.N + i] + fac * pv[1], s[po + 2 * g.N + i] + fac * pv[2]};
      cic_grad_gather(g, i, sa, djdd + (long long)b * g.M, mass, u);
    }
    T up = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const long long o = po + k * g.N + i;
      if (djdx) u[k] += djdx[o];
      xi[o] += u[k];
      const T q = pi[o] + fac * u[k];
      pi[o] = q;
      mx[k] = fmaxf(mx[k], abs_up<T>(q));
      up += u[k] * pv[k];
    }
    acc += (double)up;
  }
  const double r = block_sum(acc, shd);
  if (threadIdx.x == 0) part[(long long)b * gridDim.x + blockIdx.x] = r;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float m = block_max(mx[k], shf);
    if (threadIdx.x == 0) atomicMax(pimax + k * gridDim.y + b, __float_as_uint(m));
  }
}

// Forward: the displacement at an observed scale factor a between steps j and j + 1 from
// the state right after the step's gather, s(a) = s_{j+1} + (Dp_j(a) - D_{j+1}) p_{j+1/2}.
template <typename T>
__global__ void k_interp_state(const T* __restrict__ s, const T* __restrict__ p, const T* __restrict__ cf_tab,
                               T* __restrict__ out, long long n3) {
  const int b = blockIdx.y;
  const T cf = cf_tab[b];
  const long long o = (long long)b * n3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x)
    out[o + i] = s[o + i] + cf * p[o + i];
}

// theta[b][2] (Omega_m) += sum_k w[k][b] sums[k][b]: the theta terms of the observations
static __global__ void k_obs_theta(const double* __restrict__ sums, const double* __restrict__ w, int nk, int batch,
                                   double* __restrict__ theta) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double acc = 0.0;
  for (int k = 0; k < nk; ++k) acc += w[(long long)k * batch + b] * sums[(long long)k * batch + b];
  theta[5 * b + 2] += acc;
}

// delta = m acc 2^-e - 1 (no zeroing)
template <typename T>
__global__ void k_density_out(const long long* __restrict__ acc, T* __restrict__ out, long long total, T mul) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    out[i] = (T)acc[i] * mul - (T)1;
}

// J partials sum (delta - target)^2 and dJ/ddelta = 2 (delta - target) / M
template <typename T>
__global__ void __launch_bounds__(kPtclThreads)
k_mse(const T* __restrict__ dens, const T* __restrict__ tgt, T* __restrict__ grad, long long M, double* part) {
  __shared__ double shd[kPtclThreads / 32];
  const int b = blockIdx.y;
  const T* d = dens + (long long)b * M;
  const T* q = tgt + (long long)b * M;
  T* gr = grad + (long long)b * M;
  const T two_over_m = (T)(2.0 / (double)M);
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const T diff = d[i] - q[i];
    acc += (double)diff * diff;
    gr[i] = two_over_m * diff;
  }
  const double r = block_sum(acc, shd);
  if (threadIdx.x == 0) part[(long long)b * gridDim.x + blockIdx.x] = r;
}

// ------------------------------------------------------------------ lattice spectra
// Mode (i0, i1, kx) of an n^3 half spectrum from a flat index over main + side (main rows
// z-blocked by zb, spec_row).
struct Mode { int f0, f1, f2; long long off; };
__device__ __forceinline__ Mode mode_of(long long u, int n, int zb = 1) {
  Mode m;
  const long long main = (long long)n * n * (n / 2);
  if (u < main) {
    const int kx = (int)(u % (n / 2));
    const long long t = u / (n / 2);
    if (zb <= 1) {
      m.f1 = freq_of((int)(t % n), n);
      m.f0 = freq_of((int)(t / n), n);
    } else {
      const int zlo = (int)(t % zb);
      const long long t2 = t / zb;
      m.f1 = freq_of((int)(t2 % n), n);
      m.f0 = freq_of((int)(t2 / n) * zb + zlo, n);
    }
    m.f2 = kx;
  } else {
    const long long v = u - main;
    m.f1 = freq_of((int)(v % n), n);
    m.f0 = freq_of((int)(v / n), n);
    m.f2 = n / 2;
  }
  m.off = u;
  return m;
}
__device__ __forceinline__ int nyq_zero(int f, int n, bool last) { return last ? (f == n / 2 ? 0 : f) : (f == -n / 2 ? 0 : f); }

// s1^_c = B_c Omega, B_c = i k_c / k^2 sqrt(P / l_p^3) / n^3 (Sec. 2.1, Eqs. 3-6).  With
// amp = null the amplitude is the constant `unit` (the 2LPT s2 from the source spectrum).
template <typename T>
__global__ void k_za_mul(const cx_t<T>* __restrict__ om, cx_t<T>* o0, cx_t<T>* o1, cx_t<T>* o2, int n,
                         const T* __restrict__ amp, int maxn2, T inv_kf, long long is, T unit) {
  using C = cx_t<T>;
  const int b = blockIdx.y;
  const long long tot = spec_len_cx(n);
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < tot; u += (long long)gridDim.x * blockDim.x) {
    const Mode m = mode_of(u, n);
    const int n2 = m.f0 * m.f0 + m.f1 * m.f1 + m.f2 * m.f2;
    const C v = om[b * is + u];
    const T base = n2 ? (amp ? amp[(long long)b * (maxn2 + 1) + n2] : unit) * inv_kf / (T)n2 : (T)0;
    const int fc[3] = {nyq_zero(m.f0, n, false), nyq_zero(m.f1, n, false), nyq_zero(m.f2, n, true)};
    C* outs[3] = {o0, o1, o2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T sc = (T)fc[c] * base;
      outs[c][b * is + u] = cmake<C>(-v.y * sc, v.x * sc);  // i v sc
    }
  }
}

// Omega_bar = sum_c conj(B_c) S_c (+ acc, the 2LPT part, when given);  theta partials
// sum_k w Re[conj(Omega_bar) Omega] dlnP_j / 2.  With amp = null the amplitude is the
// constant `unit` and no partials are taken (hdlnp = null): the transpose of the 2LPT
// source -> s2 map.
template <typename T>
__global__ void __launch_bounds__(kPtclThreads)
k_za_adj_mul(const cx_t<T>* s0, const cx_t<T>* s1, const cx_t<T>* s2, const cx_t<T>* __restrict__ om,
             const cx_t<T>* acc_in, cx_t<T>* out, int n, const T* __restrict__ amp, T unit,
             const double* __restrict__ hdlnp, int maxn2, T inv_kf, long long is,
             double* part /* [5][batch][grid] */) {
  using C = cx_t<T>;
  __shared__ double shd[kPtclThreads / 32];
  const int b = blockIdx.y;
  const long long tot = spec_len_cx(n);
  double acc[5] = {0, 0, 0, 0, 0};
  const C* ins[3] = {s0, s1, s2};
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < tot; u += (long long)gridDim.x * blockDim.x) {
    const Mode m = mode_of(u, n);
    const int n2 = m.f0 * m.f0 + m.f1 * m.f1 + m.f2 * m.f2;
    const T base = n2 ? (amp ? amp[(long long)b * (maxn2 + 1) + n2] : unit) * inv_kf / (T)n2 : (T)0;
    const int fc[3] = {nyq_zero(m.f0, n, false), nyq_zero(m.f1, n, false), nyq_zero(m.f2, n, true)};
    C r = acc_in ? acc_in[b * is + u] : cmake<C>(0, 0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const C v = ins[c][b * is + u];
      const T sc = (T)fc[c] * base;
      r = cadd(r, cmake<C>(v.y * sc, -v.x * sc));  // -i v sc
    }
    out[b * is + u] = r;
    if (!hdlnp) continue;
    const C w = om[b * is + u];
    const double re = (double)r.x * w.x + (double)r.y * w.y;
    const double wt = (m.f2 == 0 || m.f2 == n / 2) ? 1.0 : 2.0;
#pragma unroll
    for (int j = 0; j < 5; ++j) acc[j] += wt * re * hdlnp[((long long)b * 5 + j) * (maxn2 + 1) + n2];
  }
  if (!hdlnp) return;
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const double r = block_sum(acc[j], shd);
    if (threadIdx.x == 0) part[((long long)j * gridDim.y + b) * gridDim.x + blockIdx.x] = r;
  }
}

// ------------------------------------------------------------ 2LPT (Sec. 2.1, Eqs. 2-4)
// The Hessian pairs (i, j) of the first-order potential: group 0 the diagonal ones
// (00, 11, 22), group 1 the mixed ones (01, 02, 12).
__device__ __forceinline__ void lpt_pair(int group, int q, int& i, int& j) {
  i = group ? (q == 2 ? 1 : 0) : q;
  j = group ? (q == 0 ? 1 : 2) : q;
}

// Hessian spectra phi_ij^ = (i k_i)(i k_j)(-1/k^2) delta1^ = k_i k_j / k^2 amp Omega
// (laplacian phi = delta1, Eq. 4), each i k_c zeroed on the Nyquist plane of axis c, for
// the three pairs of `group`; amp = sqrt(P / l_p^3) / n^3 per |n|^2.
template <typename T>
__global__ void k_lpt_hess(const cx_t<T>* __restrict__ om, cx_t<T>* o0, cx_t<T>* o1, cx_t<T>* o2, int n,
                           const T* __restrict__ amp, int maxn2, long long is, int group) {
  using C = cx_t<T>;
  const int b = blockIdx.y;
  const long long tot = spec_len_cx(n);
  C* outs[3] = {o0, o1, o2};
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < tot; u += (long long)gridDim.x * blockDim.x) {
    const Mode m = mode_of(u, n);
    const int n2 = m.f0 * m.f0 + m.f1 * m.f1 + m.f2 * m.f2;
    const C v = om[b * is + u];
    const T base = n2 ? amp[(long long)b * (maxn2 + 1) + n2] / (T)n2 : (T)0;
    const int fc[3] = {nyq_zero(m.f0, n, false), nyq_zero(m.f1, n, false), nyq_zero(m.f2, n, true)};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      int i, j;
      lpt_pair(group, q, i, j);
      const T sc = (T)(fc[i] * fc[j]) * base;
      outs[q][b * is + u] = cmake<C>(v.x * sc, v.y * sc);
    }
  }
}

// The 2LPT source S = sum_{i<j} (phi_ii phi_jj - phi_ij^2) (Eq. 4) from the real Hessian
// components r0..r2 of `group`: group 0 writes phi_00 phi_11 + phi_00 phi_22 +
// phi_11 phi_22, group 1 subtracts phi_01^2 + phi_02^2 + phi_12^2.
template <typename T>
__global__ void k_lpt_source(const T* __restrict__ r0, const T* __restrict__ r1, const T* __restrict__ r2,
                             long long ris, long long N, T* src, long long sis, int group) {
  const int b = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const T h0 = r0[b * ris + i], h1 = r1[b * ris + i], h2 = r2[b * ris + i];
    T* o = src + b * sis + i;
    if (group == 0)
      *o = h0 * h1 + h0 * h2 + h1 * h2;
    else
      *o = *o - (h0 * h0 + h1 * h1 + h2 * h2);
  }
}

// Transpose of the source at each point, in place over the Hessian components of
// `group`: phi_bar = dS/dphi S_bar, i.e. phi_bar_ii = S_bar sum_{j != i} phi_jj (group 0)
// and phi_bar_ij = -2 phi_ij S_bar (group 1).
template <typename T>
__global__ void k_lpt_source_adj(T* r0, T* r1, T* r2, long long ris, long long N, const T* __restrict__ sbar,
                                 long long sis, int group) {
  const int b = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const T h0 = r0[b * ris + i], h1 = r1[b * ris + i], h2 = r2[b * ris + i];
    const T sb = sbar[b * sis + i];
    if (group == 0) {
      r0[b * ris + i] = (h1 + h2) * sb;
      r1[b * ris + i] = (h0 + h2) * sb;
      r2[b * ris + i] = (h0 + h1) * sb;
    } else {
      r0[b * ris + i] = (T)-2 * h0 * sb;
      r1[b * ris + i] = (T)-2 * h1 * sb;
      r2[b * ris + i] = (T)-2 * h2 * sb;
    }
  }
}

// Transpose of Omega -> phi_ij (real even multipliers k_i k_j / k^2 amp): the spectra
// i0..i2 of the Hessian adjoints of `group` summed into acc (group 0 overwrites acc).
template <typename T>
__global__ void k_lpt_hess_adj(const cx_t<T>* __restrict__ i0, const cx_t<T>* __restrict__ i1,
                               const cx_t<T>* __restrict__ i2, cx_t<T>* acc, int n, const T* __restrict__ amp,
                               int maxn2, long long is, int group) {
  using C = cx_t<T>;
  const int b = blockIdx.y;
  const long long tot = spec_len_cx(n);
  const C* ins[3] = {i0, i1, i2};
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < tot; u += (long long)gridDim.x * blockDim.x) {
    const Mode m = mode_of(u, n);
    const int n2 = m.f0 * m.f0 + m.f1 * m.f1 + m.f2 * m.f2;
    const T base = n2 ? amp[(long long)b * (maxn2 + 1) + n2] / (T)n2 : (T)0;
    const int fc[3] = {nyq_zero(m.f0, n, false), nyq_zero(m.f1, n, false), nyq_zero(m.f2, n, true)};
    C r = group ? acc[b * is + u] : cmake<C>(0, 0);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      int i, j;
      lpt_pair(group, q, i, j);
      const T sc = (T)(fc[i] * fc[j]) * base;
      const C v = ins[q][b * is + u];
      r = cadd(r, cmake<C>(v.x * sc, v.y * sc));
    }
    acc[b * is + u] = r;
  }
}

// Second-order terms of the initial state: s += D2 s2, p += G_D2 s2, s2 kept for the
// adjoint's Omega_m terms (Sec. 2.1, Eq. 2).
template <typename T>
__global__ void k_ic_state2(const T* __restrict__ r0, const T* __restrict__ r1, const T* __restrict__ r2,
                            long long ris, long long N, const T* __restrict__ d2, const T* __restrict__ gd2, T* s2,
                            T* s, T* p) {
  const int b = blockIdx.y;
  const T* rs[3] = {r0 + b * ris, r1 + b * ris, r2 + b * ris};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T v = rs[c][i];
      const long long o = (long long)b * 3 * N + c * N + i;
      s2[o] = v;
      s[o] = s[o] + d2[b] * v;
      p[o] = p[o] + gd2[b] * v;
    }
  }
}

// s1 from the lattice C2R outputs; s = D1 s1, p = G_D s1
template <typename T>
__global__ void k_ic_state(const T* __restrict__ r0, const T* __restrict__ r1, const T* __restrict__ r2, long long ris,
                           long long N, const T* __restrict__ d1, const T* __restrict__ gd, T* s1, T* s, T* p) {
  const int b = blockIdx.y;
  const T* rs[3] = {r0 + b * ris, r1 + b * ris, r2 + b * ris};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T v = rs[c][i];
      const long long o = (long long)b * 3 * N + c * N + i;
      if (s1) s1[o] = v;
      if (s) s[o] = d1[b] * v;
      if (p) p[o] = gd[b] * v;
    }
  }
}

// Fixed-point state from the initial state: U = round(s / l 2^kFixES), W = round(p / l
// 2^kFixEP), and s, p replaced by their shadows
template <typename T>
__global__ void k_fix_init(T* __restrict__ s, T* __restrict__ p, FixState<T> fx, T to_u, long long n3) {
  const int b = blockIdx.y;
  const long long o0 = (long long)b * n3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x) {
    const long long o = o0 + i;
    const long long U = to_fixed<T>(mul_rn<T>(s[o], to_u));
    const long long W = to_fixed<T>(mul_rn<T>(p[o], fx.to_w));
    fx.u[o] = U;
    fx.w[o] = W;
    s[o] = mul_rn<T>(fix_to_real<T>(U), fx.from_u);
    p[o] = mul_rn<T>(fix_to_real<T>(W), fx.from_w);
  }
}

// sbar = D1 xi + G_D pi into the lattice FFT inputs; partials of xi.s1 and pi.s1
template <typename T>
__global__ void __launch_bounds__(kPtclThreads)
k_ic_adj_prep(const T* __restrict__ xi, const T* __restrict__ pi, const T* __restrict__ s1, long long N,
              const T* __restrict__ d1, const T* __restrict__ gd, T* w0, T* w1, T* w2, long long wis,
              double* part_xs, double* part_ps) {
  __shared__ double shd[kPtclThreads / 32];
  const int b = blockIdx.y;
  T* ws[3] = {w0 + b * wis, w1 + b * wis, w2 + b * wis};
  double axs = 0, aps = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long o = (long long)b * 3 * N + c * N + i;
      const T x = xi[o], q = pi[o], u = s1[o];
      ws[c][i] = d1[b] * x + gd[b] * q;
      axs += (double)x * u;
      aps += (double)q * u;
    }
  }
  const double r1 = block_sum(axs, shd);
  const double r2 = block_sum(aps, shd);
  if (threadIdx.x == 0) {
    part_xs[(long long)b * gridDim.x + blockIdx.x] = r1;
    part_ps[(long long)b * gridDim.x + blockIdx.x] = r2;
  }
}

// Fixed-order sum of `count` partials for each instance: out[b] = sum_i part[b][i]
static __global__ void k_sum_partials(const double* __restrict__ part, int count, double* out, double scale) {
  __shared__ double shd[8];
  const int b = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += part[(long long)b * count + i];
  const double r = block_sum(acc, shd);
  if (threadIdx.x == 0) out[b] = r * scale;
}

// dJ/dtheta (Eq. 51): time-stepping terms (Omega_m only), initial-condition growth terms
// and the P_lin derivative terms.  sums: per instance the already reduced scalars.
struct ThetaIn {
  const double* step_pa;   // pi.a at step j, instance b: step_pa[j * step_stride + b]
  const double* step_xp;   // xi.p at step j: step_xp[j * step_stride + b]
  const double* w_pa;      // weight of pi.a: w_pa[j * batch + b]
  const double* w_xp;      // weight of xi.p
  const double* xs;        // [batch]   xi_0 . s1
  const double* ps;        // [batch]   pi_0 . s1
  const double* dlp;       // [5][batch]
  const double* dd1;       // [batch]   dD1(a0)/dOm
  const double* dgd;       // [batch]   dG_D(a0)/dOm
  const double* xs2;       // [batch]   xi_0 . s2   (2LPT; null at first order)
  const double* ps2;       // [batch]   pi_0 . s2
  const double* dd2;       // [batch]   dD2(a0)/dOm
  const double* dgd2;      // [batch]   dG_D2(a0)/dOm
  int nstep1, batch, step_stride;
};
static __global__ void k_final_theta(ThetaIn in, double* out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= in.batch) return;
  double g = 0.0;
  for (int j = 0; j < in.nstep1; ++j) {
    const long long o = (long long)j * in.step_stride + b;
    const long long w = (long long)j * in.batch + b;
    g += in.step_pa[o] * in.w_pa[w] + in.step_xp[o] * in.w_xp[w];
  }
  g += in.xs[b] * in.dd1[b] + in.ps[b] * in.dgd[b];
  if (in.xs2) g += in.xs2[b] * in.dd2[b] + in.ps2[b] * in.dgd2[b];
  for (int j = 0; j < 5; ++j) out[5 * b + j] = in.dlp[j * in.batch + b] + (j == 2 ? g : 0.0);
}

// ------------------------------------------------------------- power spectrum
// Shell-averaged power of a half spectrum (summary statistic of Sec. 2.4): bin b holds the
// modes with b <= |n| < b + 1; off-plane modes count twice (for their conjugates).  The
// sums are exact int64 fixed point with a per-bin scale from a first max pass, so the
// result does not depend on the order of the additions.
__device__ __forceinline__ int isqrt_floor(int v) {
  int r = (int)sqrtf((float)v);
  while (r * r > v) --r;
  while ((r + 1) * (r + 1) <= v) ++r;
  return r;
}

template <typename T>
__global__ void k_power_max(const cx_t<T>* __restrict__ spec, int n, long long is, int nb, unsigned* pmax) {
  const int b = blockIdx.y;
  const long long tot = spec_len_cx(n);
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < tot; u += (long long)gridDim.x * blockDim.x) {
    const Mode m = mode_of(u, n, spec_zb(n));
    const int bin = isqrt_floor(m.f0 * m.f0 + m.f1 * m.f1 + m.f2 * m.f2);
    if (bin >= nb) continue;
    const cx_t<T> v = spec[b * is + u];
    const double w = (m.f2 == 0 || m.f2 == n / 2) ? 1.0 : 2.0;
    const double p = w * ((double)v.x * v.x + (double)v.y * v.y);
    atomicMax(pmax + b * nb + bin, __float_as_uint(__double2float_ru(p)));
  }
}

template <typename T>
__global__ void k_power_acc(const cx_t<T>* __restrict__ spec, int n, long long is, int nb, const int* __restrict__ e,
                            unsigned long long* acc, unsigned long long* cnt, unsigned long long* ksum) {
  const int b = blockIdx.y;
  const long long tot = spec_len_cx(n);
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < tot; u += (long long)gridDim.x * blockDim.x) {
    const Mode m = mode_of(u, n, spec_zb(n));
    const int n2 = m.f0 * m.f0 + m.f1 * m.f1 + m.f2 * m.f2;
    const int bin = isqrt_floor(n2);
    if (bin >= nb) continue;
    const cx_t<T> v = spec[b * is + u];
    const int w = (m.f2 == 0 || m.f2 == n / 2) ? 1 : 2;
    const double p = w * ((double)v.x * v.x + (double)v.y * v.y);
    atomicAdd(acc + b * nb + bin, (unsigned long long)__double2ll_rn(ldexp(p, e[b * nb + bin])));
    if (b == 0) {
      atomicAdd(cnt + bin, (unsigned long long)w);
      atomicAdd(ksum + bin, (unsigned long long)__double2ll_rn(w * sqrt((double)n2) * 1048576.0));
    }
  }
}

// per-bin exponent: sum over <= 2^lgM modes of values < 2^E stays below 2^62
static __global__ void k_power_exponents(const unsigned* __restrict__ pmax, int* e, int count, int lgM) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float mx = __uint_as_float(pmax[i]);
  e[i] = (mx > 0.f && isfinite(mx)) ? min(62 - lgM - (ilogbf(mx) + 1), 1000) : 0;
}

static __global__ void k_power_final(const unsigned long long* acc, const unsigned long long* cnt,
                                     const unsigned long long* ksum, const int* e, int nb, int batch, double vol_m2,
                                     double kf, double* pk, double* kmean, double* nmodes) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb * batch) return;
  const int bin = i % nb;
  const double c = (double)cnt[bin];
  pk[i] = c > 0 ? vol_m2 * ldexp((double)(long long)acc[i], -e[i]) / c : 0.0;
  if (i < nb) {
    if (kmean) kmean[bin] = c > 0 ? kf * ldexp((double)(long long)ksum[bin], -20) / c : 0.0;
    if (nmodes) nmodes[bin] = c;
  }
}

// Objective on the shell power (summary statistic of Sec. 2.4), one thread per instance:
// J = sum_b w_b (P_b - T_b)^2 in fixed bin order, and the per-bin factor of its density
// cotangent g_b = 2 w_b (P_b - T_b) 2 V / (M^2 C_b) (0 for empty bins).
static __global__ void k_power_loss(const double* __restrict__ pk, const double* __restrict__ nmodes,
                                    const double* __restrict__ tgt, const double* __restrict__ w, int nb, int batch,
                                    double two_v_m2, double* loss, double* g) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double j = 0.0;
  for (int i = 0; i < nb; ++i) {
    const long long o = (long long)b * nb + i;
    const double d = pk[o] - tgt[o];
    j += w[o] * d * d;
    const double c = nmodes[i];
    g[o] = c > 0 ? 2.0 * w[o] * d * two_v_m2 / c : 0.0;
  }
  loss[b] = j;
}

// Cotangent spectrum g_b(|n|) delta^ in place over the half spectrum (bins b < nb, 0 beyond);
// its unnormalised inverse transform is dJ/d delta (d P_b / d delta(x) is 2V / (M^2 C_b)
// times the inverse transform of delta^ restricted to shell b).
template <typename T>
__global__ void k_power_grad(cx_t<T>* spec, int n, long long is, int nb, const double* __restrict__ g) {
  const int b = blockIdx.y;
  const long long tot = spec_len_cx(n);
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < tot; u += (long long)gridDim.x * blockDim.x) {
    const Mode m = mode_of(u, n, spec_zb(n));
    const int bin = isqrt_floor(m.f0 * m.f0 + m.f1 * m.f1 + m.f2 * m.f2);
    const T f = bin < nb ? (T)g[(long long)b * nb + bin] : (T)0;
    cx_t<T> v = spec[b * is + u];
    v.x *= f;
    v.y *= f;
    spec[b * is + u] = v;
  }
}

// numpy rfftn layout <-> main + side spectrum layout (for the FFT operator entry point)
template <typename T>
__global__ void k_spec_to_std(const cx_t<T>* __restrict__ spec, cx_t<T>* __restrict__ out, int n, long long total) {
  const int h = n / 2 + 1;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < total; u += (long long)gridDim.x * blockDim.x) {
    const long long per = (long long)n * n * h;
    const long long b = u / per, r = u % per;
    const int k = (int)(r % h);
    const long long row = r / h;
    const cx_t<T>* base = spec + b * spec_len_cx(n);
    const long long mrow = spec_row(n, spec_lzb(n), (int)(row / n), (int)(row % n));
    out[u] = k < n / 2 ? base[mrow * (n / 2) + k] : base[spec_main_len(n) + row];
  }
}
template <typename T>
__global__ void k_std_to_spec(const cx_t<T>* __restrict__ in, cx_t<T>* __restrict__ spec, int n, long long total) {
  const int h = n / 2 + 1;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < total; u += (long long)gridDim.x * blockDim.x) {
    const long long per = (long long)n * n * h;
    const long long b = u / per, r = u % per;
    const int k = (int)(r % h);
    const long long row = r / h;
    cx_t<T>* base = spec + b * spec_len_cx(n);
    const long long mrow = spec_row(n, spec_lzb(n), (int)(row / n), (int)(row % n));
    if (k < n / 2) base[mrow * (n / 2) + k] = in[u];
    else base[spec_main_len(n) + row] = in[u];
  }
}

}  // namespace pmgb
