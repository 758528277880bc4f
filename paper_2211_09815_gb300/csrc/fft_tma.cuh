// TMA-staged, double-buffered persistent column passes of the 3-D FFT (y and z axes of
// the main half spectrum), templated on the real type.
//
// One CTA per SM loops over column tiles (TC sequences x L elements).  A single thread
// issues the tensor-memory-accelerator loads of the next tile into a free slot of a
// shared-memory ring (cp.async.bulk.tensor, completion on an mbarrier) while the CTA works
// on the current tile, so HBM reads of tile t+1 overlap the radix stages of tile t.  The
// last radix stage writes its tile into shared memory and the same thread stores it with
// TMA (cp.async.bulk.tensor from shared memory, bulk async-groups).
//   KIND 0: in-place column FFT of up to four buffers (direction DIR)
//   KIND 1: z FFT of delta^, 2 inverse z FFTs: of -i k_0 G delta^ (z force) and of
//           G delta^ (shared by the y and x force components; -i k_1 and -i k_2 are
//           constant along a z column)
//   KIND 2: z FFTs of P_0 and of V = i (k_1 P_1 + k_2 P_2), accumulated as
//           G (i k_0 P_0 + V), 1 inverse z FFT (adjoint psi)
//   KIND 3: inverse y of U: IFFT(U) and IFFT(-i k_1 U)
//   KIND 4: forward y of P_1 and P_2 into V = i (k_1 Y(P_1) + k_2 Y(P_2))
// Every mbarrier wait is bounded: on timeout the CTA records an error flag, waits (again
// bounded) for its own copies in flight, and returns.
#pragma once
#include <type_traits>

#include <cuda.h>

#include "fft.cuh"

namespace pmgb {

struct TmaMaps { CUtensorMap m[4]; };

template <typename T> struct TmaJob {
  cx_t<T>* out[4];     // KIND 0: the buffers; 1: z force, U; 2: psi; 3: y force (U's buffer),
                       // x force before -i k_2; 4: V (P_1's buffer)
  int nbuf;            // KIND 0: buffers in the launch
  int zaxis;           // 0: y pass, 1: z pass
  int batch;
  const T* coef;       // Green's function coefficient per instance (KIND 1, 2)
  const T* dtab;       // deconvolution table or null
  int* err;            // device error flag (mbarrier timeout)
  int first_wait;      // spin limit of each CTA's first wait (< 0: the normal limit)
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false (and the error flag set) if the phase does not complete within
// `spins` polls (negative: 2^24 polls, far beyond any tile load)
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int* err, int spins = -1) {
  const long long lim = spins < 0 ? (1LL << 24) : (long long)spins;
  for (long long i = 0; i < lim; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  if (err) *(volatile int*)err = 1;
  return false;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, unsigned long long* bar, int c0, int c1,
                                            int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, unsigned long long* bar, int c0, int c1,
                                            int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
      "[%7];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(c4), "r"(smem_u32(bar))
      : "memory");
}

// TMA store of a shared-memory box into the tensor (bulk async-group of the issuing
// thread); the writers of the box execute fence_proxy_async and a barrier first
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int c0, int c1, int c2, int c3) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];"
               ::"l"(reinterpret_cast<unsigned long long>(map)), "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2),
                 "r"(c3)
               : "memory");
}
__device__ __forceinline__ void tma_store_5d(const CUtensorMap* map, const void* src, int c0, int c1, int c2, int c3,
                                             int c4) {
  asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5, %6}], [%1];"
               ::"l"(reinterpret_cast<unsigned long long>(map)), "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2),
                 "r"(c3), "r"(c4)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory sources of this thread's committed stores have been read
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// ... all but the most recently committed one
__device__ __forceinline__ void bulk_wait_read_but1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
// this thread's committed stores are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// dense [L][TC] tile (TMA writes rows back to back)
template <typename C, int LD>
struct DenseTile {
  C* p;
  __device__ __forceinline__ C ld(int row, int c) const { return p[row * LD + c]; }
  __device__ __forceinline__ void st(int row, int c, C v) const { p[row * LD + c] = v; }
  static constexpr bool kLinear = true;
  static constexpr int kLD = LD;
  __device__ __forceinline__ C* ptr(int row, int c) const { return p + row * LD + c; }
  __host__ __device__ static constexpr int delta(int d) { return d; }
};

// Tiles of the staged passes: 64 KB of TC columns (at least 128-byte rows of a TMA box for
// L >= 512), transformed with the two-stage radix-32 plans at L = 512 and 1024, where a
// third stage would add a read and a write of the whole tile in shared memory.
template <typename T, int L> constexpr int tma_tc() {
  return L >= 512 ? 65536 / (L * (int)sizeof(cx_t<T>)) : ColTile<T, L>::TC;
}
// Radix plan of a TMA column pass: the two-stage radix-32 plans, except for the fused
// adjoint z pass (KIND 2), which takes the three-stage radix-16 plan where its thread count
// (one radix-16 butterfly per thread) fits in a block: twice the warps per SM for a pass
// of three transforms per tile bound by instruction latency, not by HBM (measured 9%
// faster at 1024^3).  The fused z force keeps radix 32: its register hand-off saves a
// shared-memory round trip and a Green's function per element (radix 16 was 21% slower
// without the hand-off and 11% slower with it, forward 16-8-8 into inverse 8-8-16), and
// the y split and merge (KIND 3, 4) were 5% slower with radix 16.
template <typename T, int L, int KIND> struct TmaPlanOf {
  static constexpr bool kR16 = KIND == 2 && tma_tc<T, L>() * L / Plan<L>::RMAX <= 512;
  using type = std::conditional_t<kR16, Plan<L>, Plan2<L>>;
};
template <typename T, int L, class PL = Plan2<L>> struct TmaTile {
  using P = PL;
  static constexpr int TC = tma_tc<T, L>();
  static constexpr int NT = TC * L / P::RMAX;
  static constexpr int LD = TC;
  static_assert(NT <= 512 && (L / 2) % TC == 0, "TMA tile shape");
  static constexpr int RB = L < 256 ? L : 256;                  // rows per TMA box
  static constexpr int TILE = L * TC;                            // complex elements per tile
  static constexpr int BYTES = TILE * (int)sizeof(cx_t<T>);
  static constexpr int W = (int)sizeof(cx_t<T>) / 8;              // int64 words per complex
  static constexpr int ZB = spec_zb(L);                          // z blocking of the main rows
};

// Green's function data for a z-pass column (kx, y), as in the unstaged fused kernels.
template <typename T, int N>
struct ZCol {
  T coef, d12;
  int n12, f1, f2;
  const T* dtab;
  __device__ __forceinline__ T g(int f0) const {
    const int n2 = f0 * f0 + n12;
    if (n2 == 0) return (T)0;
    T v = coef * d12 / (T)n2;
    if (dtab) v *= dtab[f0 < 0 ? f0 + N : f0];
    return v;
  }
  __device__ __forceinline__ int fc(int comp, int f0) const {
    if (comp == 0) return f0 == -N / 2 ? 0 : f0;
    if (comp == 1) return f1 == -N / 2 ? 0 : f1;
    return f2;   // main array: kx < N/2, never the Nyquist plane
  }
};

// z pass, force: multiplier of the inverse transform of output `mode`:
//   0: -i k_0 G (the z component), 1: G (shared by the y and x components, whose -i k_1
//   and -i k_2 are constant along a z column and are applied in the y and x passes)
template <typename T, int N, int LD>
struct DenseMulSrc {
  const cx_t<T>* p;
  ZCol<T, N> z;
  int mode;
  __device__ __forceinline__ cx_t<T> ld(int row, int c) const { return apply(p[row * LD + c], row, z, mode); }
  static __device__ __forceinline__ cx_t<T> apply(cx_t<T> v, int row, const ZCol<T, N>& z, int mode) {
    const int f0 = freq_of(row, N);
    const T g = z.g(f0);
    if (mode == 1) return cmake<cx_t<T>>(v.x * g, v.y * g);
    const T s = (T)z.fc(0, f0) * g;
    return cmake<cx_t<T>>(v.y * s, -v.x * s);
  }
};
// z pass, adjoint: the last forward stage of input `mode` into the accumulator:
//   0: A = conj(-i k_0 G) v = i k_0 G v;  1: A += G v (the input already carries
//   i (k_1 P_1 + k_2 P_2), formed in the y pass)
template <typename T, int N, int LD>
struct DenseAccDst {
  cx_t<T>* p;
  ZCol<T, N> z;
  int mode;
  __device__ __forceinline__ void st(int row, int c, cx_t<T> v) const {
    const int f0 = freq_of(row, N);
    const T g = z.g(f0);
    cx_t<T>* q = p + row * LD + c;
    if (mode == 1) {
      *q = cadd(*q, cmake<cx_t<T>>(v.x * g, v.y * g));
    } else {
      const T s = (T)z.fc(0, f0) * g;
      *q = cmake<cx_t<T>>(-v.y * s, v.x * s);
    }
  }
};
// signed frequency along a column with the Nyquist row zeroed (derivative rule)
template <int N> __device__ __forceinline__ int fc_row(int row) {
  const int f = freq_of(row, N);
  return f == -N / 2 ? 0 : f;
}
// y pass, inverse split: source -i k_1 v of the y component
template <typename T, int N, int LD>
struct YMulSrc {
  const cx_t<T>* p;
  __device__ __forceinline__ cx_t<T> ld(int row, int c) const {
    const cx_t<T> v = p[row * LD + c];
    const T s = (T)fc_row<N>(row);
    return cmake<cx_t<T>>(v.y * s, -v.x * s);
  }
};
// y pass, forward merge: A = i k_1 Y(P_1), then out = A + i k_2 Y(P_2) written to HBM
template <typename T, int N, int LD>
struct YAccDst {
  cx_t<T>* p;
  __device__ __forceinline__ void st(int row, int c, cx_t<T> v) const {
    const T s = (T)fc_row<N>(row);
    p[row * LD + c] = cmake<cx_t<T>>(-v.y * s, v.x * s);
  }
};
template <typename T, int LD>
struct YMergeDst {  // in place in the accumulator tile
  cx_t<T>* acc;
  T k2;             // x frequency of the column
  __device__ __forceinline__ void st(int row, int c, cx_t<T> v) const {
    cx_t<T>* q = acc + row * LD + c;
    const cx_t<T> a = *q;
    *q = cmake<cx_t<T>>(a.x - v.y * k2, a.y + v.x * k2);
  }
};

template <typename T, int L, int DIR, int KIND>
__global__ void __launch_bounds__(TmaTile<T, L, typename TmaPlanOf<T, L, KIND>::type>::NT, 1)
k_cols_tma(const __grid_constant__ TmaMaps maps, const __grid_constant__ TmaMaps omaps,
           const __grid_constant__ TmaJob<T> job, int tiles_per_buf, const cx_t<T>* __restrict__ tw) {
  using C = cx_t<T>;
  using TT = TmaTile<T, L, typename TmaPlanOf<T, L, KIND>::type>;
  constexpr int N = L;
  constexpr int NCG = (N / 2) / TT::TC;            // column groups per row of the main array
  constexpr int NL = (KIND == 2 || KIND == 4) ? 2 : 1;   // loads per work item
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // TMA destinations must be 128-byte aligned: round the dynamic base up (1 KiB slack)
  C* ring0 = reinterpret_cast<C*>((reinterpret_cast<unsigned long long>(smem_raw) + 1023ull) & ~1023ull);
  // ring slots of the prefetched tiles: three for the plain passes (no work tile), two
  // and a work tile for the others
  constexpr int NSLOT = KIND == 0 ? 3 : 2;
  auto slot = [&](int q) { return ring0 + (q % NSLOT) * TT::TILE; };
  C* work = ring0 + 2 * TT::TILE;
  // twiddle table of the length-L transform: the fused passes copy it into shared memory
  // once per CTA (measured faster there; the plain column passes read it through L1)
  C* tws = ring0 + 3 * TT::TILE;
  if constexpr (KIND != 0)
    for (int m = threadIdx.x; m < L; m += blockDim.x) tws[m] = __ldg(tw + m);
  const SmemTw<C> stw{tws};
  __shared__ unsigned long long bars[NSLOT];
  const int items = KIND == 0 ? job.nbuf * tiles_per_buf : tiles_per_buf;
  const int my_items = blockIdx.x < (unsigned)items ? (items - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int nq = my_items * NL;
  if (threadIdx.x == 0) {
    for (int k = 0; k < NSLOT; ++k) mbar_init(&bars[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // load q of this CTA -> (work item, component)
  auto decode = [&](int q, int& item, int& comp) {
    item = blockIdx.x + (q / NL) * gridDim.x;
    comp = q % NL;
  };
  auto issue = [&](int q) {
    int item, comp;
    decode(q, item, comp);
    const int buf = KIND == 0 ? item / tiles_per_buf : comp;
    const int u = KIND == 0 ? item % tiles_per_buf : item;
    const int kxg = u % NCG, o = (u / NCG) % N, b = u / (NCG * N);
    C* dst = slot(q);
    unsigned long long* bar = &bars[q % NSLOT];
    fence_proxy_async();
    mbar_expect_tx(bar, TT::BYTES);
    // 5-D view of the main array: (kx words, z mod ZB, y, z / ZB, instance)
#pragma unroll
    for (int r = 0; r < L / TT::RB; ++r) {
      if (job.zaxis)
        tma_load_5d(dst + r * TT::RB * TT::LD, &maps.m[buf], bar, kxg * TT::TC * TT::W, 0, o, r * (TT::RB / TT::ZB),
                    b);
      else
        tma_load_5d(dst + r * TT::RB * TT::LD, &maps.m[buf], bar, kxg * TT::TC * TT::W, o % TT::ZB, r * TT::RB,
                    o / TT::ZB, b);
    }
  };
  // Results leave by TMA stores from shared memory.  KIND 0: three slots, so the slot
  // refilled at the top of an iteration was stored two iterations earlier.  KIND 1 and 3
  // (two outputs: the work tile, then the input's own slot): the next load is issued after
  // the first output, when the previous tile's stores out of that slot have long been
  // read.  KIND 2 and 4 store only the work tile.
  constexpr bool kStore = true;
  auto store = [&](const CUtensorMap* map, const C* src, int kxg, int o, int b) {
#pragma unroll
    for (int r = 0; r < L / TT::RB; ++r) {
      if (job.zaxis)
        tma_store_5d(map, src + r * TT::RB * TT::LD, kxg * TT::TC * TT::W, 0, o, r * (TT::RB / TT::ZB), b);
      else
        tma_store_5d(map, src + r * TT::RB * TT::LD, kxg * TT::TC * TT::W, o % TT::ZB, r * TT::RB, o / TT::ZB, b);
    }
    bulk_commit();
  };
  if (threadIdx.x == 0 && nq > 0) issue(0);
  const int c = threadIdx.x % TT::TC;
  for (int q = 0; q < nq; ++q) {
    if (threadIdx.x == 0) {
      if (KIND == 0) {
        bulk_wait_read_but1();
        if (q + 1 < nq) issue(q + 1);
      } else if (KIND == 3) {
        bulk_wait_read_but1();   // the work tile: its store is older than the newest
      } else if ((KIND == 2 || KIND == 4) && q + 1 < nq) {
        issue(q + 1);   // the ring slots are never store sources here
      }
    }
    if (!mbar_wait(&bars[q % NSLOT], (q / NSLOT) & 1, job.err, q == 0 ? job.first_wait : -1)) {
      // drain this CTA's loads in flight (bounded) before it exits: the load of slot q,
      // and the next one where it was issued before this wait (KIND 0, 2, 4); then the
      // committed stores
      if (threadIdx.x == 0) {
        mbar_wait(&bars[q % NSLOT], (q / NSLOT) & 1, nullptr);
        if ((KIND == 0 || KIND == 2 || KIND == 4) && q + 1 < nq)
          mbar_wait(&bars[(q + 1) % NSLOT], ((q + 1) / NSLOT) & 1, nullptr);
        if (kStore) bulk_wait_all();
      }
      return;
    }
    int item, comp;
    decode(q, item, comp);
    const int u = KIND == 0 ? item % tiles_per_buf : item;
    const int kxg = u % NCG, o = (u / NCG) % N, b = u / (NCG * N);
    C* cur = slot(q);
    DenseTile<C, TT::LD> t{cur};
    if constexpr (KIND == 0) {
      fft_tile<T, L, TT::TC, TT::NT, DIR, typename TT::P>(t, t, t, tw);
      fence_proxy_async();
      __syncthreads();
      if (threadIdx.x == 0) store(&maps.m[item / tiles_per_buf], cur, kxg, o, b);
    } else if constexpr (KIND == 1 || KIND == 2) {
      ZCol<T, N> zc;
      zc.f1 = freq_of(o, N);
      zc.f2 = kxg * TT::TC + c;
      zc.n12 = zc.f1 * zc.f1 + zc.f2 * zc.f2;
      zc.coef = job.coef[b];
      zc.dtab = job.dtab;
      zc.d12 = job.dtab ? job.dtab[zc.f1 < 0 ? zc.f1 + N : zc.f1] * job.dtab[zc.f2] : (T)1;
      DenseTile<C, TT::LD> wt{work};
      if constexpr (KIND == 1 && TT::P::S == 2) {
        // two-stage plan (RA, RB): the forward transform's last stage leaves the spectrum
        // in registers, item j holding rows j + RA r (r < RB) -- exactly the inputs of the
        // first stage of an inverse transform planned as (RB, RA) -- so both inverse
        // transforms start from registers instead of a shared-memory round trip
        constexpr int RA = TT::P::R0, RB = TT::P::R1, TC = TT::TC, NT = TT::NT;
        constexpr int PER = TC * (L / RB) / NT;
        stage<T, L, TC, NT, RA, 1, -1>(t, t, stw);
        __syncthreads();
        C x[PER][RB];
        T gz[PER][RB];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
          const int j = (threadIdx.x + i * NT) / TC;      // j < L / RB = RA
#pragma unroll
          for (int r = 0; r < RB; ++r) x[i][r] = cur[(j + r * RA) * TT::LD + c];
#pragma unroll
          for (int r = 1; r < RB; ++r) x[i][r] = cmul(x[i][r], twiddle<-1>(stw, r * j));   // jm = j, L/(RA RB) = 1
          dft<RB, -1>(x[i]);                                // x[i][r] = X[j + RA r]
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          // the other ring slot and the work tile are no longer read by the previous
          // tile's stores: refill the slot
          bulk_wait_read_all();
          if (q + 1 < nq) issue(q + 1);
        }
        __syncthreads();   // the work tile is written below, after that wait
        // the Green's function of each row, shared by both outputs (one division per element)
#pragma unroll
        for (int i = 0; i < PER; ++i) {
          const int j = (threadIdx.x + i * NT) / TC;
#pragma unroll
          for (int r = 0; r < RB; ++r) {
            const int f0 = freq_of(j + RA * r, N);
            const T gv = zc.g(f0);
            x[i][r] = cmake<C>(x[i][r].x * gv, x[i][r].y * gv);      // G X
            gz[i][r] = (T)zc.fc(0, f0);                               // k_0 (Nyquist row 0)
          }
        }
#pragma unroll
        for (int mode = 0; mode < 2; ++mode) {
          // mode 0: -i k_0 G X (z force) -> work; mode 1: G X (U) -> the ring slot
          C* dst = mode == 0 ? work : cur;
#pragma unroll
          for (int i = 0; i < PER; ++i) {
            const int j = (threadIdx.x + i * NT) / TC;
            C y[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r)
              y[r] = mode == 1 ? x[i][r] : cmake<C>(x[i][r].y * gz[i][r], -x[i][r].x * gz[i][r]);
            dft<RB, +1>(y);                                  // inverse stage 1 (NS = 1)
#pragma unroll
            for (int r = 0; r < RB; ++r) dst[(j * RB + r) * TT::LD + c] = y[r];
          }
        }
        __syncthreads();
        stage<T, L, TC, NT, RA, RB, +1>(wt, wt, stw);        // inverse stage 2 of the z force
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) store(&omaps.m[0], work, kxg, o, b);
        stage<T, L, TC, NT, RA, RB, +1>(t, t, stw);          // and of U
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) store(&omaps.m[1], cur, kxg, o, b);
      } else if constexpr (KIND == 1) {
        fft_tile<T, L, TT::TC, TT::NT, -1, typename TT::P>(t, t, t, stw);
        __syncthreads();
        if (threadIdx.x == 0) {
          // the other ring slot and the work tile are no longer read by the previous
          // tile's stores: refill the slot (the work tile is first written after the
          // barrier inside the next radix stage)
          bulk_wait_read_all();
          if (q + 1 < nq) issue(q + 1);
        }
        // z force: -i k_0 G T -> work -> out[0]
        DenseMulSrc<T, N, TT::LD> src0{cur, zc, 0};
        fft_tile<T, L, TT::TC, TT::NT, +1, typename TT::P>(src0, wt, wt, stw);
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) store(&omaps.m[0], work, kxg, o, b);
        // U: G T -> in place in the ring slot -> out[1]
        DenseMulSrc<T, N, TT::LD> src1{cur, zc, 1};
        fft_tile<T, L, TT::TC, TT::NT, +1, typename TT::P>(src1, t, t, stw);
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) store(&omaps.m[1], cur, kxg, o, b);
      } else {
        // the accumulator (work tile) is first written by the last radix stage, after the
        // barriers of the earlier ones: the previous item's store must have read it
        if (comp == 0 && threadIdx.x == 0) bulk_wait_read_all();
        DenseAccDst<T, N, TT::LD> acc{work, zc, comp};
        fft_tile<T, L, TT::TC, TT::NT, -1, typename TT::P>(t, t, acc, stw);
        if (comp == 1) {
          __syncthreads();
          fft_tile<T, L, TT::TC, TT::NT, +1, typename TT::P>(wt, wt, wt, stw);
          fence_proxy_async();
          __syncthreads();
          if (threadIdx.x == 0) store(&omaps.m[0], work, kxg, o, b);
        }
      }
    } else if constexpr (KIND == 3) {
      // inverse y of the shared x/y force transform U: IFFT(U) -> out[1] (the x component
      // before its -i k_2), IFFT(-i k_1 U) -> out[0] (the y component, in place)
      DenseTile<C, TT::LD> wt{work};
      fft_tile<T, L, TT::TC, TT::NT, +1, typename TT::P>(t, wt, wt, stw);
      fence_proxy_async();
      __syncthreads();
      if (threadIdx.x == 0) {
        store(&omaps.m[1], work, kxg, o, b);
        bulk_wait_read_but1();   // the other slot's store (previous tile) has been read
        if (q + 1 < nq) issue(q + 1);
      }
      YMulSrc<T, N, TT::LD> src{cur};
      fft_tile<T, L, TT::TC, TT::NT, +1, typename TT::P>(src, t, t, stw);
      fence_proxy_async();
      __syncthreads();
      if (threadIdx.x == 0) store(&omaps.m[0], cur, kxg, o, b);
    } else {
      // forward y of the adjoint's x and y sums: out[0] = i (k_1 Y(P_1) + k_2 Y(P_2))
      if (comp == 0) {
        if (threadIdx.x == 0) bulk_wait_read_all();   // the previous item's store of the work tile
        YAccDst<T, N, TT::LD> acc{work};
        fft_tile<T, L, TT::TC, TT::NT, -1, typename TT::P>(t, t, acc, stw);
      } else {
        YMergeDst<T, TT::LD> dst{work, (T)(kxg * TT::TC + c)};
        fft_tile<T, L, TT::TC, TT::NT, -1, typename TT::P>(t, t, dst, stw);
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) store(&omaps.m[0], work, kxg, o, b);
      }
    }
    __syncthreads();
  }
  if (kStore && threadIdx.x == 0) bulk_wait_all();
}

}  // namespace pmgb
