// Hand-written batched 3-D real FFT for the particle-mesh force (Sec. 2.2, Eq. 11):
// device building blocks.
//
// A length-L complex DFT of a tile of TC independent sequences is done as a Stockham
// auto-sort FFT with mixed radices (<= 16).  Each stage: every thread loads the R
// inputs of its butterfly, applies the stage twiddles, does an R-point DFT in registers
// and stores the R outputs at their Stockham positions.  A tile in shared memory is
// laid out [L][LD] with the sequence index innermost, so that for column passes a warp's
// loads and stores touch consecutive addresses.  The unstaged column passes read the
// first stage straight from global memory and write the last one straight back; the
// TMA-staged ones (fft_tma.cuh) work on tiles in shared memory; the x passes load rows
// into shared memory with coalesced reads first.
#pragma once
#include "common.cuh"

namespace pmgb {

// Radix plan for a length-L transform: stages R0 (first) .. R2, all <= 16.
template <int L> struct Plan;
template <> struct Plan<2>    { static constexpr int S = 1, R0 = 2,  R1 = 1, R2 = 1, RMAX = 2; };
template <> struct Plan<4>    { static constexpr int S = 1, R0 = 4,  R1 = 1, R2 = 1, RMAX = 4; };
template <> struct Plan<8>    { static constexpr int S = 1, R0 = 8,  R1 = 1, R2 = 1, RMAX = 8; };
template <> struct Plan<16>   { static constexpr int S = 1, R0 = 16, R1 = 1, R2 = 1, RMAX = 16; };
template <> struct Plan<32>   { static constexpr int S = 2, R0 = 8,  R1 = 4, R2 = 1, RMAX = 8; };
template <> struct Plan<64>   { static constexpr int S = 2, R0 = 8,  R1 = 8, R2 = 1, RMAX = 8; };
template <> struct Plan<128>  { static constexpr int S = 2, R0 = 16, R1 = 8, R2 = 1, RMAX = 16; };
template <> struct Plan<256>  { static constexpr int S = 2, R0 = 16, R1 = 16, R2 = 1, RMAX = 16; };
template <> struct Plan<512>  { static constexpr int S = 3, R0 = 8,  R1 = 8, R2 = 8, RMAX = 8; };
template <> struct Plan<1024> { static constexpr int S = 3, R0 = 16, R1 = 8, R2 = 8, RMAX = 16; };

// Two-stage plans (radix 32) for the long column transforms, where shared memory, not
// HBM, limits the three-stage plans: each stage reads and writes the whole tile once.
template <int L> struct Plan2 : Plan<L> {};
template <> struct Plan2<512>  { static constexpr int S = 2, R0 = 32, R1 = 16, R2 = 1, RMAX = 32; };
template <> struct Plan2<1024> { static constexpr int S = 2, R0 = 32, R1 = 32, R2 = 1, RMAX = 32; };

// cos(2 pi m / 32): exact values of the 32nd roots of unity (the 16th roots are the even m).
__host__ __device__ constexpr double cos32(int m) {
  m &= 31;
  const int a = m > 16 ? 32 - m : m;   // cos(2 pi m / 32) = cos(2 pi (32 - m) / 32)
  const int b = a > 8 ? 16 - a : a;    // cos(pi - x) = -cos(x)
  const double v = b == 0 ? 1.0 : b == 1 ? 0.98078528040323044913 : b == 2 ? 0.92387953251128675613
                 : b == 3 ? 0.83146961230254523708 : b == 4 ? 0.70710678118654752440
                 : b == 5 ? 0.55557023301960222474 : b == 6 ? 0.38268343236508977173
                 : b == 7 ? 0.19509032201612826785 : 0.0;
  return a > 8 ? -v : v;
}
__host__ __device__ constexpr double sin32(int m) { return cos32(m - 8); }

// v <- v * exp(DIR * 2 pi i k / R), R <= 32.  k is a compile-time index of the unrolled
// butterflies, so the multiples of pi/4 resolve to their exact forms at compile time: a
// swap and negation for +-i and -1 (a product with a zero cosine would stay in the code:
// x * 0 is not folded under IEEE rules), two products for the diagonals.
template <int R, int DIR, typename C>
__device__ __forceinline__ C root_mul(C v, int k) {
  using T = decltype(v.x);
  static_assert(R <= 32, "roots of unity up to order 32");
  const int m = (k * (32 / R)) & 31;
  if (m == 0) return v;
  if (m == 16) return cmake<C>(-v.x, -v.y);
  if (m == 8) return DIR > 0 ? cmake<C>(-v.y, v.x) : cmake<C>(v.y, -v.x);       // DIR i
  if (m == 24) return DIR > 0 ? cmake<C>(v.y, -v.x) : cmake<C>(-v.y, v.x);      // -DIR i
  if ((m & 3) == 0) {   // m = 4, 12, 20, 28: (+-1 +- i) / sqrt(2)
    const T h = (T)0.70710678118654752440;
    const T c = m == 4 || m == 28 ? (T)1 : (T)-1;
    const T s = (T)(DIR * (m < 16 ? 1 : -1));
    return cmake<C>((c * v.x - s * v.y) * h, (s * v.x + c * v.y) * h);
  }
  const T c = (T)cos32(m), s = (T)(DIR * sin32(m));
  return cmake<C>(v.x * c - v.y * s, v.x * s + v.y * c);
}

// In-register R-point DFT, natural order in and out: X_k = sum_r v_r exp(DIR 2 pi i r k / R)
template <int R, int DIR, typename C>
__device__ __forceinline__ void dft(C (&v)[R]) {
  if constexpr (R == 1) {
    return;
  } else if constexpr (R == 2) {
    const C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else {
    C e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) { e[i] = v[2 * i]; o[i] = v[2 * i + 1]; }
    dft<R / 2, DIR>(e);
    dft<R / 2, DIR>(o);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      const C t = (k == 0) ? o[k] : root_mul<R, DIR>(o[k], k);
      v[k] = cadd(e[k], t);
      v[k + R / 2] = csub(e[k], t);
    }
  }
}

// exp(DIR 2 pi i m / L) from the table w[m] = exp(-2 pi i m / L), read through the
// read-only data cache, or from a copy in shared memory (SmemTw)
template <int DIR, typename C>
__device__ __forceinline__ C twiddle(const C* __restrict__ w, int m) {
  C t = __ldg(w + m);
  if (DIR > 0) t.y = -t.y;
  return t;
}
template <typename C> struct SmemTw { const C* p; };
template <int DIR, typename C>
__device__ __forceinline__ C twiddle(const SmemTw<C>& w, int m) {
  C t = w.p[m];
  if (DIR > 0) t.y = -t.y;
  return t;
}

// ---------------------------------------------------------------- tile accessors
// Shared-memory row of tile element (row, c): one padding row is inserted after every 16
// rows, so that the rows 16 apart that the first radix-16 stage stores in one warp
// instruction fall into different halves of the 32 banks.
__host__ __device__ constexpr int skew_rows(int rows) { return rows + (rows >> 4); }
__device__ __forceinline__ int srow(int row) { return row + (row >> 4); }

template <typename C, int LD>
struct SmemTile {
  C* p;
  __device__ __forceinline__ C ld(int row, int c) const { return p[srow(row) * LD + c]; }
  __device__ __forceinline__ void st(int row, int c, C v) const { p[srow(row) * LD + c] = v; }
  // Linear access for the radix stages: the rows base + d that a butterfly touches never
  // carry out of the low four bits of base (see stage()), so the skewed row of base + d is
  // srow(base) + delta(d) with a compile-time delta.
  static constexpr bool kLinear = true;
  static constexpr int kLD = LD;
  __device__ __forceinline__ C* ptr(int row, int c) const { return p + srow(row) * LD + c; }
  __host__ __device__ static constexpr int delta(int d) { return d + (d >> 4); }
};

// accessors without a linear form (global sequences, multipliers) take the generic path
template <class X, class = void> struct IsLinear { static constexpr bool value = false; };
template <class X> struct IsLinear<X, decltype(void(X::kLinear))> { static constexpr bool value = X::kLinear; };

// one sequence per thread in global memory: element `row` at p[row * es]
template <typename C>
struct GlobalSeq {
  C* p;
  long long es;
  bool valid;
  __device__ __forceinline__ C ld(int row, int) const {
    if (!valid) return cmake<C>(0, 0);
    return p[(long long)row * es];
  }
  __device__ __forceinline__ void st(int row, int, C v) const {
    if (valid) p[(long long)row * es] = v;
  }
};

// One Stockham radix-R stage over TC sequences of length L, NT threads.
// NS = product of the radices already applied.  Loads all of the thread's inputs, syncs,
// then stores, so source and destination may be the same shared-memory tile.
template <typename T, int L, int TC, int NT, int R, int NS, int DIR, class Src, class Dst, class TW>
__device__ __forceinline__ void stage(const Src& src, const Dst& dst, const TW& tw) {
  using C = cx_t<T>;
  constexpr int ITEMS = TC * (L / R);
  constexpr int PER = ITEMS / NT;
  static_assert(PER * NT == ITEMS, "work items must divide evenly");
  C v[PER][R];
  const int c = threadIdx.x % TC;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int j = (threadIdx.x + i * NT) / TC;
    // rows j + r L/R: j < L/R, and L/R is a power of two, so the low four bits of j plus
    // those of r L/R never carry (a linear tile reads them at compile-time offsets)
    if constexpr (IsLinear<Src>::value) {
      const C* p = src.ptr(j, c);
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = p[Src::delta(r * (L / R)) * Src::kLD];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = src.ld(j + r * (L / R), c);
    }
    if constexpr (NS > 1) {
      const int jm = j % NS;
#pragma unroll
      for (int r = 1; r < R; ++r) v[i][r] = cmul(v[i][r], twiddle<DIR>(tw, r * jm * (L / (NS * R))));
    }
    dft<R, DIR>(v[i]);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int j = (threadIdx.x + i * NT) / TC;
    const int jd = (j / NS) * NS * R + (j % NS);
    // rows jd + r NS: jd = (multiple of NS R) + (j mod NS); for NS >= 16 the step is a
    // multiple of 16, for NS < 16 (a power of two) the offsets stay inside the 16-row block
    if constexpr (IsLinear<Dst>::value) {
      C* p = dst.ptr(jd, c);
#pragma unroll
      for (int r = 0; r < R; ++r) p[Dst::delta(r * NS) * Dst::kLD] = v[i][r];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) dst.st(jd + r * NS, c, v[i][r]);
    }
  }
}

// Full length-L DFT of a tile: src -> (mid) -> dst.  `mid` must be a shared tile.  P: the
// radix plan (Plan<L> or Plan2<L>).
template <typename T, int L, int TC, int NT, int DIR, class P = Plan<L>, class Src, class Mid, class Dst, class TW>
__device__ __forceinline__ void fft_tile(const Src& src, const Mid& mid, const Dst& dst, const TW& tw) {
  if constexpr (P::S == 1) {
    stage<T, L, TC, NT, P::R0, 1, DIR>(src, dst, tw);
  } else if constexpr (P::S == 2) {
    stage<T, L, TC, NT, P::R0, 1, DIR>(src, mid, tw);
    __syncthreads();
    stage<T, L, TC, NT, P::R1, P::R0, DIR>(mid, dst, tw);
  } else {
    stage<T, L, TC, NT, P::R0, 1, DIR>(src, mid, tw);
    __syncthreads();
    stage<T, L, TC, NT, P::R1, P::R0, DIR>(mid, mid, tw);
    __syncthreads();
    stage<T, L, TC, NT, P::R2, P::R0 * P::R1, DIR>(mid, dst, tw);
  }
}

// Tile shapes.  Column passes: TC sequences of length L in one tile of <= BYTES,
// NT = TC * L / RMAX threads (each thread holds RMAX values), NT <= 512.
template <typename T, int L, int BYTES = 65536> struct ColTile {
  static constexpr int RMAX = Plan<L>::RMAX;
  static constexpr int TC0 = BYTES / (L * (int)sizeof(cx_t<T>));
  static constexpr int TC1 = TC0 > 256 ? 256 : TC0;
  static constexpr int TCMAXNT = 512 * RMAX / L;
  static constexpr int TC2 = TC1 < TCMAXNT ? TC1 : TCMAXNT;
  static constexpr int TC = TC2 < 1 ? 1 : TC2;
  static constexpr int NT = TC * L / RMAX;
  static constexpr int LD = TC;
  static constexpr int SMEM = skew_rows(L) * LD * (int)sizeof(cx_t<T>);
};
// Fused z passes keep two tiles of the column-pass shape.
template <typename T, int L> using FusedTile = ColTile<T, L, 65536>;
// Row passes (x axis): TR rows of L = n/2 complex values, tile padded to LD = TR + 1 so
// that the transposing row loads do not collide in shared-memory banks.  Rows of 512
// points run the two-stage radix-32 plan on 64 KB tiles (one shared-memory round trip less
// than three radix-8 stages); shorter rows the three-stage plans on 32 KB tiles.
template <typename T, int L> struct RowTile {
  using P = Plan2<L>;
  static constexpr int RMAX = P::RMAX;
  static constexpr int TR0 = (RMAX == 32 ? 65536 : 32768) / (L * (int)sizeof(cx_t<T>));
  static constexpr int TR1 = TR0 > 128 ? 128 : TR0;
  static constexpr int TRMAXNT = 512 * RMAX / L;
  static constexpr int TR2 = TR1 < TRMAXNT ? TR1 : TRMAXNT;
  // a tile never spans two instances: TR divides the n^2 = 4 L^2 rows of one mesh
  static constexpr int TR3 = TR2 < 4 * L * L ? TR2 : 4 * L * L;
  static constexpr int TR = TR3 < 1 ? 1 : TR3;
  // at most 256 threads (measured faster than one radix item per thread at L = 512)
  static constexpr int NT0 = TR * L / RMAX;
  static constexpr int NT = NT0 > 256 ? 256 : NT0;
  static_assert(NT >= 1 && TR * L % RMAX == 0, "row tile needs whole work items");
  static constexpr int LD = TR + 1;
  static constexpr int SMEM = skew_rows(L) * LD * (int)sizeof(cx_t<T>);
};

}  // namespace pmgb
