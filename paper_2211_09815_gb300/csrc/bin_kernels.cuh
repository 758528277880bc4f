// Deterministic CIC assignment without global atomics on the mesh ("owner computes").
//
// Every step the particles are binned by the mesh tile that holds their cell (tiles of
// tx x ty x tz cells, x = array axis 2 fastest).  A bin is a tile and a class of three
// bits telling whether the cell lies on the tile's last layer along x, y, z: only those
// particles' CIC clouds reach into the next tile.  One CTA per tile then pulls the
// particles of its own bins and the reaching classes of its seven lower neighbours, and
// sums the weights (and in the adjoint pi_c times the weights) of the corners that land
// in its tile in 64-bit fixed point in shared memory.  Every contribution is rounded to
// fixed point on its own, exactly as in a global fixed-point deposit, so the sums are
// exact and independent of the order of the particles.  The CTA then writes the real
// meshes (delta and pi_c) once, in the working precision.
//
// Binning: a count (warp-aggregated integer atomics on an L2-resident array; inside a
// simulation step the gather kernels count the bins of the positions they have just
// written, count_bin in pm_kernels.cuh), an exclusive scan, and a fill that writes each
// particle's record (cell fractions, cell within its tile, and in the adjoint the scaled
// pi) in bin order, so that a tile's CTA reads its particles as contiguous runs.
#pragma once
#include "pm_kernels.cuh"

namespace pmgb {

// Warp-uniform loop over the work indices of this block's warps: every lane of a warp
// takes the same number of iterations, so that the warp-wide match below sees all lanes.
template <typename T>
__global__ void __launch_bounds__(kPtclThreads)
k_bin_count(Geo<T> g, BinGeo bg, const T* __restrict__ s, unsigned* __restrict__ count, unsigned* __restrict__ keys) {
  const int b = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const T* sb = s + (long long)b * 3 * g.N;
  unsigned* cb = count + (long long)b * bg.nkeys;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long w0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); w0 < g.N; w0 += stride) {
    const long long w = w0 + lane;
    const bool valid = w < g.N;
    unsigned key = 0xFFFFFFFFu;
    if (valid) {
      const long long i = particle_of(g, w);
      const T sv[3] = {sb[i], sb[g.N + i], sb[2 * g.N + i]};
      int cell[3];
      T t[3];
      cic_cell(g, i, sv, cell, t);
      key = bin_key(bg, cell);
      keys[(long long)b * g.N + i] = key;
    }
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
    if (valid && lane == __ffs(peers) - 1) atomicAdd(cb + key, (unsigned)__popc(peers));
  }
}

// local cell coordinates of a particle inside its own tile, 10 bits per axis
__device__ __forceinline__ unsigned pack_local(const BinGeo& bg, const int c[3]) {
  return ((unsigned)c[0] & ((1u << bg.lz) - 1)) << 20 | ((unsigned)c[1] & ((1u << bg.ly) - 1)) << 10 |
         ((unsigned)c[2] & ((1u << bg.lx) - 1));
}
template <typename T> __device__ __forceinline__ T bits_to_real(unsigned u);
template <> __device__ __forceinline__ float bits_to_real<float>(unsigned u) { return __uint_as_float(u); }
template <> __device__ __forceinline__ double bits_to_real<double>(unsigned u) { return __longlong_as_double((long long)u); }
template <typename T> __device__ __forceinline__ unsigned real_to_bits(T v);
template <> __device__ __forceinline__ unsigned real_to_bits<float>(float v) { return __float_as_uint(v); }
template <> __device__ __forceinline__ unsigned real_to_bits<double>(double v) { return (unsigned)__double_as_longlong(v); }

// rec0[pos] = (t_0, t_1, t_2, local cell bits); with pi, rec1[pos] = (pi_c 2^e_c, 0)
template <typename T, int NQ>
__global__ void __launch_bounds__(kPtclThreads)
k_bin_fill(Geo<T> g, BinGeo bg, const T* __restrict__ s, const T* __restrict__ pi, const int* __restrict__ e_pi,
           const unsigned* __restrict__ keys, unsigned* __restrict__ cursor, V4<T>* __restrict__ rec0,
           V4<T>* __restrict__ rec1) {
  const int b = blockIdx.y;
  const int lane = threadIdx.x & 31;
  unsigned* cb = cursor + (long long)b * bg.nkeys;
  const T* sb = s + (long long)b * 3 * g.N;
  T sp[3] = {0, 0, 0};
  if constexpr (NQ == 4) {
#pragma unroll
    for (int c = 0; c < 3; ++c) sp[c] = pow2i<T>(e_pi[c * gridDim.y + b]);
  }
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long w0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); w0 < g.N; w0 += stride) {
    const long long w = w0 + lane;
    const bool valid = w < g.N;
    unsigned key = 0xFFFFFFFFu;
    // every load of the particle first (key, position, pi), then the cursor atomic
    V4<T> r0{0, 0, 0, 0}, r1{0, 0, 0, 0};
    if (valid) {
      const long long i = particle_of(g, w);
      key = keys[(long long)b * g.N + i];
      const T sv[3] = {sb[i], sb[g.N + i], sb[2 * g.N + i]};
      if constexpr (NQ == 4) {
        const T* pb = pi + (long long)b * 3 * g.N;
        r1 = V4<T>{pb[i] * sp[0], pb[g.N + i] * sp[1], pb[2 * g.N + i] * sp[2], (T)0};
      }
      int cell[3];
      T t[3];
      cic_cell(g, i, sv, cell, t);
      r0 = V4<T>{t[0], t[1], t[2], bits_to_real<T>(pack_local(bg, cell))};
    }
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
    const int leader = __ffs(peers) - 1;
    unsigned pos = 0;
    if (valid && lane == leader) pos = atomicAdd(cb + key, (unsigned)__popc(peers));
    pos = __shfl_sync(0xFFFFFFFFu, pos, leader);
    if (valid) {
      pos += __popc(peers & ((1u << lane) - 1u));
      rec0[pos] = r0;
      if constexpr (NQ == 4) rec1[pos] = r1;
    }
  }
}

// Exclusive scan of n counts in three launches: blocks of 2048 elements, the block totals
// (one block), the add-back.  The scan also clears the counts for the next binning and
// initialises the fill cursors.
constexpr int kScanBlock = 2048;
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* sh, unsigned* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;   // 256 threads
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned t = lane < 8 ? sh[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < 8) sh[lane] = t;
  }
  __syncthreads();
  const unsigned base = w > 0 ? sh[w - 1] : 0u;
  *total = sh[7];
  __syncthreads();
  return base + x - v;
}

static __global__ void __launch_bounds__(256) k_scan_blocks(unsigned* __restrict__ count, unsigned* __restrict__ start,
                                                            unsigned* __restrict__ sums, long long n) {
  __shared__ unsigned sh[8];
  const long long base = (long long)blockIdx.x * kScanBlock + threadIdx.x * 8;
  unsigned v[8], tsum = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k] = base + k < n ? count[base + k] : 0u;
    tsum += v[k];
  }
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (base + k < n) count[base + k] = 0u;
  unsigned total;
  unsigned run = block_excl_scan(tsum, sh, &total);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (base + k < n) start[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

static __global__ void __launch_bounds__(256) k_scan_sums(unsigned* __restrict__ sums, int nblocks) {
  __shared__ unsigned sh[8];
  unsigned carry = 0;
  for (int first = 0; first < nblocks; first += kScanBlock) {
    const int base = first + threadIdx.x * 8;
    unsigned v[8], tsum = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      v[k] = base + k < nblocks ? sums[base + k] : 0u;
      tsum += v[k];
    }
    unsigned total;
    unsigned run = carry + block_excl_scan(tsum, sh, &total);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (base + k < nblocks) sums[base + k] = run;
      run += v[k];
    }
    carry += total;
  }
}

static __global__ void k_scan_add(unsigned* __restrict__ start, unsigned* __restrict__ cursor,
                                  const unsigned* __restrict__ sums, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned v = start[i] + sums[i / kScanBlock];
    start[i] = v;
    cursor[i] = v;
  }
}

// The 20 particle ranges a tile pulls: (offset d of the source tile below, first class).
// d = 0: the tile's own 8 bins as one range; d != 0: each class containing the bits of d,
// one bin each.  Packed 3 bits per range.
constexpr unsigned long long pack3(const int (&v)[20]) {
  unsigned long long r = 0;
  for (int k = 0; k < 20; ++k) r |= (unsigned long long)v[k] << (3 * k);
  return r;
}
constexpr int kRangeDv[20] = {0, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 4, 4, 4, 4, 5, 5, 6, 6, 7};
constexpr int kRangeCv[20] = {0, 1, 3, 5, 7, 2, 3, 6, 7, 3, 7, 4, 5, 6, 7, 5, 7, 6, 7, 7};
constexpr unsigned long long kRangeD = pack3(kRangeDv);
constexpr unsigned long long kRangeC = pack3(kRangeCv);

// Exact 64-bit addition into a shared accumulator kept as two 32-bit words: the low word
// takes a native 32-bit atomic add whose returned old value gives the carry, the high word
// the high part plus that carry.  Each addition is exact mod 2^64, so the final pair holds
// the exact sum in any order (64-bit shared atomics are several times slower).
__device__ __forceinline__ void smem_add64(unsigned* lo, unsigned* hi, unsigned vl, unsigned vh) {
  const unsigned old = atomicAdd(lo, vl);
  const unsigned h = vh + (old + vl < old ? 1u : 0u);
  if (h) atomicAdd(hi, h);
}
// the exact sum (two words) in the working precision, correctly rounded; sums that fit in
// 32 bits take one hardware conversion
template <typename T> __device__ __forceinline__ T words_to_real(unsigned lo, unsigned hi);
template <> __device__ __forceinline__ float words_to_real<float>(unsigned lo, unsigned hi) {
  if (hi == 0u) return __uint2float_rn(lo);
  if (hi == 0xFFFFFFFFu && (lo >> 31)) return __int2float_rn((int)lo);
  return ll2f_rn((long long)(((unsigned long long)hi << 32) | lo));
}
template <> __device__ __forceinline__ double words_to_real<double>(unsigned lo, unsigned hi) {
  return (double)(long long)(((unsigned long long)hi << 32) | lo);
}

// Accumulation of one tile (shared by the unfused and the fused deposit): the ranges of
// the tile's own bins and the reaching classes of its seven lower neighbours, each CIC
// corner that lands in the tile rounded to fixed point and added exactly.  acc: low words
// [NQ][cells], then high words [NQ][cells] (zeroed here).
template <typename T, int NQ>
__device__ __forceinline__ void pull_accumulate(const BinGeo& bg, const V4<T>* __restrict__ rec0,
                                                const V4<T>* __restrict__ rec1, const unsigned* __restrict__ start,
                                                int e_d, int b, int tile, unsigned* acc, unsigned* rbeg,
                                                unsigned* rpre) {
  const int T2 = tile & (bg.ntx - 1), T1 = (tile / bg.ntx) & (bg.nty - 1), T0 = tile / (bg.ntx * bg.nty);
  const int cells = 1 << (bg.lx + bg.ly + bg.lz);
  // the first warp reads the range bounds (one lane per range) before the accumulator is
  // cleared, so that their latency overlaps the clearing
  const int ri = threadIdx.x;
  unsigned ra = 0, re = 0;
  if (ri < 20) {
    const int d = (int)((kRangeD >> (3 * ri)) & 7u), c0 = (int)((kRangeC >> (3 * ri)) & 7u);
    const int S2 = (T2 - (d & 1)) & (bg.ntx - 1);
    const int S1 = (T1 - ((d >> 1) & 1)) & (bg.nty - 1);
    const int S0 = (T0 - ((d >> 2) & 1)) & (bg.ntz - 1);
    const long long key0 = (long long)b * bg.nkeys + ((long long)(S0 * bg.nty + S1) * bg.ntx + S2) * 8 + c0;
    ra = start[key0];
    re = start[key0 + (d == 0 ? 8 : 1)];
  }
  for (int k = threadIdx.x; k < NQ * cells / 2; k += blockDim.x) reinterpret_cast<uint4*>(acc)[k] = make_uint4(0, 0, 0, 0);
  unsigned* hacc = acc + NQ * cells;
  if (threadIdx.x < 32) {
    const unsigned len = re - ra;
    if (ri < 20) rbeg[ri] = ra;
    unsigned x = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (ri >= o) x += y;
    }
    if (ri < 21) rpre[ri] = x - len;   // exclusive prefix; rpre[20] = total
  }
  __syncthreads();
  const T sd = pow2i<T>(e_d);
  const unsigned total = rpre[20];
  const unsigned mx = (1u << bg.lx) - 1, my = (1u << bg.ly) - 1, mz = (1u << bg.lz) - 1;
  for (unsigned f = threadIdx.x; f < total; f += blockDim.x) {
    int r = 0;
    while (f >= rpre[r + 1]) ++r;
    const unsigned d = (unsigned)((kRangeD >> (3 * r)) & 7u);
    const unsigned pos = rbeg[r] + (f - rpre[r]);
    const V4<T> r0 = rec0[pos];
    const T t[3] = {r0.x, r0.y, r0.z};
    const unsigned packed = real_to_bits<T>(r0.w);
    const int l0 = (int)(packed >> 20), l1 = (int)((packed >> 10) & 1023u), l2 = (int)(packed & 1023u);
    const unsigned cls = (unsigned)((unsigned)l2 == mx) | ((unsigned)((unsigned)l1 == my) << 1) |
                         ((unsigned)((unsigned)l0 == mz) << 2);
    T pv[3] = {0, 0, 0};
    if constexpr (NQ == 4) {
      const V4<T> r1 = rec1[pos];
      pv[0] = r1.x;
      pv[1] = r1.y;
      pv[2] = r1.z;
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      // corner e (bit 2: axis 0, bit 1: axis 1, bit 0: axis 2) crosses into the next tile
      // along an axis iff the cell is on the tile's last layer there and the corner is the
      // upper one; it lands in this CTA's tile iff those crossings equal d
      const unsigned carry = cls & (unsigned)e;
      if (carry != d) continue;
      const int a0 = (d & 4u) ? 0 : l0 + ((e >> 2) & 1);
      const int a1 = (d & 2u) ? 0 : l1 + ((e >> 1) & 1);
      const int a2 = (d & 1u) ? 0 : l2 + (e & 1);
      const int loc = (((a0 << bg.ly) + a1) << bg.lx) + a2;
      const T w = ((e & 4) ? t[0] : (T)1 - t[0]) * ((e & 2) ? t[1] : (T)1 - t[1]) * ((e & 1) ? t[2] : (T)1 - t[2]);
      unsigned vl, vh;
      fixed_words<T>(w * sd, vl, vh);
      smem_add64(acc + loc, hacc + loc, vl, vh);
      if constexpr (NQ == 4) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          fixed_words<T>(pv[c] * w, vl, vh);
          smem_add64(acc + (1 + c) * cells + loc, hacc + (1 + c) * cells + loc, vl, vh);
        }
      }
    }
  }
  __syncthreads();
}

// One CTA per tile (grid: tiles x instances; tile x extent >= 4, outputs 16-byte aligned).
// NQ = 1: delta; NQ = 4: delta and the three
// pi sums.  Outputs: delta = m acc 2^-e_d - 1 into dout (instance stride dis), pi_c =
// acc 2^-e_c into p0..p2 (instance stride pis).  Dynamic shared memory: NQ * cells * 8 B
// (low words [NQ][cells], then high words [NQ][cells]).
template <typename T, int NQ, int NT>
__global__ void __launch_bounds__(NT, NT >= 512 ? 3 : 1)
k_pull_scatter(Geo<T> g, BinGeo bg, const V4<T>* __restrict__ rec0, const V4<T>* __restrict__ rec1,
               const unsigned* __restrict__ start, int e_d, const int* __restrict__ e_pi, T mass,
               T* __restrict__ dout, long long dis, T* __restrict__ p0, T* __restrict__ p1, T* __restrict__ p2,
               long long pis) {
  extern __shared__ __align__(16) unsigned acc[];   // [2][NQ][cells]
  __shared__ unsigned rbeg[20], rpre[21];
  const int b = blockIdx.y;
  const int tile = blockIdx.x;
  const int T2 = tile & (bg.ntx - 1), T1 = (tile / bg.ntx) & (bg.nty - 1), T0 = tile / (bg.ntx * bg.nty);
  const int cells = 1 << (bg.lx + bg.ly + bg.lz);
  pull_accumulate<T, NQ>(bg, rec0, rec1, start, e_d, b, tile, acc, rbeg, rpre);
  const unsigned* hacc = acc + NQ * cells;
  const unsigned mx = (1u << bg.lx) - 1, my = (1u << bg.ly) - 1;
  const T md = mass * pow2i<T>(-e_d);
  T mp[3] = {0, 0, 0};
  if constexpr (NQ == 4) {
#pragma unroll
    for (int c = 0; c < 3; ++c) mp[c] = pow2i<T>(-e_pi[c * gridDim.y + b]);
  }
  // four neighbouring x cells per thread (tile x extent >= 4): 16-byte shared loads of
  // both words, one vector store per quantity
  const long long tile_base = ((long long)(T0 << bg.lz) * g.nm + (T1 << bg.ly)) * g.nm + (T2 << bg.lx);
  for (int k = threadIdx.x * 4; k < cells; k += blockDim.x * 4) {
    const int a2 = k & (int)mx, a1 = (k >> bg.lx) & (int)my, a0 = k >> (bg.lx + bg.ly);
    const long long cell = tile_base + ((long long)a0 * g.nm + a1) * g.nm + a2;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const uint4 lo = *reinterpret_cast<const uint4*>(acc + q * cells + k);
      const uint4 hi = *reinterpret_cast<const uint4*>(hacc + q * cells + k);
      const T m = q == 0 ? md : mp[q - 1];
      const T a = q == 0 ? (T)-1 : (T)0;
      const V4<T> v{words_to_real<T>(lo.x, hi.x) * m + a, words_to_real<T>(lo.y, hi.y) * m + a,
                    words_to_real<T>(lo.z, hi.z) * m + a, words_to_real<T>(lo.w, hi.w) * m + a};
      T* o = q == 0 ? dout + b * dis : (q == 1 ? p0 : (q == 2 ? p1 : p2)) + b * pis;
      *reinterpret_cast<V4<T>*>(o + cell) = v;
    }
  }
}

}  // namespace pmgb
