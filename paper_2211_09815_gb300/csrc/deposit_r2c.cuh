// Tile-owner CIC deposit fused with the x pass of the real-to-complex FFT.
//
// The mesh tiles of this deposit span whole x rows (n cells) and R rows in (y, z), so the
// CTA that owns a tile holds every cell of its rows once the particles have been summed
// in shared memory.  Instead of writing the real meshes (delta, and in the adjoint the
// three pi sums) to HBM for a separate x pass to read back, the CTA converts its exact
// fixed-point sums to the working precision, transforms each of its rows along x in
// shared memory (two reals per complex, an L = n/2 point FFT, the even/odd split) and
// writes the half-spectrum rows (main and side plane) that the y and z column passes take
// next.  The sums, and so the transformed values, are the same as those of the unfused
// deposit followed by the x pass (the same rounding of every contribution, the same
// radix stages).
//
// Particle binning, ranges and accumulation are those of bin_kernels.cuh (ntx = 1: a
// tile's x neighbour is itself, so a CIC corner past x = n - 1 lands at x = 0 of the same
// tile, the periodic wrap).
#pragma once
#include "bin_kernels.cuh"
#include "fft.cuh"

namespace pmgb {

// Shape of the fused deposit for rows of n = 2L cells: R rows per tile, TC = NQ R row
// transforms, NT threads.  R is chosen so that a tile holds 2^13 (one quantity) or 2^12
// (four quantities) cells in FP32, half of that in FP64; NT gives the radix stages whole
// work items (up to 1024 threads: the shared memory of a four-quantity tile admits one
// CTA per SM, and the accumulation needs the warps).
template <typename T, int NQ, int L> struct FusedDeposit {
  static constexpr int N = 2 * L;
  static constexpr int CELLS0 = (NQ == 1 ? 8192 : 4096) / (int)(sizeof(T) / 4);
  static constexpr int R0 = CELLS0 / N;
  static constexpr int R = R0 < 1 ? 1 : R0;
  static constexpr int CELLS = N * R;
  static constexpr int TC = NQ * R;                           // row transforms per tile
  static constexpr int NT0 = TC * L / Plan<L>::RMAX;
  static constexpr int NT = NT0 > 1024 ? 1024 : NT0;   // one radix item per thread where possible
  static constexpr int LD = TC + 1;
  static constexpr int ACC_BYTES = NQ * CELLS * 8;
  static constexpr int FFT_BYTES = skew_rows(L) * LD * (int)sizeof(cx_t<T>);
  static constexpr int SMEM = ACC_BYTES > FFT_BYTES ? ACC_BYTES : FFT_BYTES;
  static constexpr int VPT = NQ * CELLS / NT;                 // values per thread in the conversion
  static_assert(VPT % 2 == 0 && NQ * CELLS % (2 * NT) == 0, "two cells (one complex) per item");
  static_assert((TC * L / Plan<L>::RMAX) % NT == 0, "radix stages need whole work items");
};

template <typename T> struct FusedOut {
  cx_t<T>* spec[4];   // half spectra of delta, pi_0, pi_1, pi_2 (main + side, instance stride spec_len_cx)
  T* dens;            // optional real delta [batch][M]
};

// One CTA per tile of FusedDeposit<T, NQ, L>::R full x rows (grid: tiles x instances).
// bg must have lx = log2(n) (one tile across x) and ly + lz = log2(R).
template <typename T, int NQ, int L>
__global__ void __launch_bounds__(FusedDeposit<T, NQ, L>::NT)
k_pull_r2c(BinGeo bg, const V4<T>* __restrict__ rec0, const V4<T>* __restrict__ rec1,
           const unsigned* __restrict__ start, int e_d, const int* __restrict__ e_pi, T mass, FusedOut<T> out,
           const cx_t<T>* __restrict__ twL, const cx_t<T>* __restrict__ twN) {
  using C = cx_t<T>;
  using FD = FusedDeposit<T, NQ, L>;
  constexpr int N = FD::N, R = FD::R, CELLS = FD::CELLS, TC = FD::TC, NT = FD::NT;
  extern __shared__ __align__(16) unsigned acc[];
  __shared__ unsigned rbeg[20], rpre[21];
  const int b = blockIdx.y;
  const int tile = blockIdx.x;
  pull_accumulate<T, NQ>(bg, rec0, rec1, start, e_d, b, tile, acc, rbeg, rpre);

  // exact sums -> working precision: delta = m acc 2^-e_d - 1, pi_c = acc 2^-e_c; two
  // neighbouring x cells (one complex of the packed row) per item, all read before the
  // shared memory is reused for the transforms
  const unsigned* hacc = acc + NQ * CELLS;
  const T md = mass * pow2i<T>(-e_d);
  T mp[3] = {0, 0, 0};
  if constexpr (NQ == 4) {
#pragma unroll
    for (int c = 0; c < 3; ++c) mp[c] = pow2i<T>(-e_pi[c * gridDim.y + b]);
  }
  const int T1 = tile % bg.nty, T0 = tile / bg.nty;   // ntx = 1
  constexpr int ITEMS = FD::VPT / 2;
  C v[ITEMS];
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const int u = 2 * (threadIdx.x + it * NT);     // flat index over [NQ][cells], even
    const int q = u / CELLS, k = u % CELLS;
    const uint2 lo = *reinterpret_cast<const uint2*>(acc + u);
    const uint2 hi = *reinterpret_cast<const uint2*>(hacc + u);
    const T m = q == 0 ? md : (q == 1 ? mp[0] : (q == 2 ? mp[1] : mp[2]));   // selects: no local array
    const T a = q == 0 ? (T)-1 : (T)0;
    v[it] = cmake<C>(words_to_real<T>(lo.x, hi.x) * m + a, words_to_real<T>(lo.y, hi.y) * m + a);
    if (q == 0 && out.dens) {
      const int r = k / N, x = k % N;
      const long long cell = ((long long)((T0 << bg.lz) + (r >> bg.ly)) * N + ((T1 << bg.ly) + (r & ((1 << bg.ly) - 1)))) * N + x;
      *reinterpret_cast<C*>(out.dens + (long long)b * N * N * N + cell) = v[it];
    }
  }
  __syncthreads();
  C* sm = reinterpret_cast<C*>(acc);
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const int u = 2 * (threadIdx.x + it * NT);
    const int q = u / CELLS, k = u % CELLS;
    const int r = k / N, j = (k % N) / 2;
    sm[srow(j) * FD::LD + q * R + r] = v[it];
  }
  __syncthreads();
  SmemTile<C, FD::LD> t{sm};
  fft_tile<T, L, TC, NT, -1>(t, t, t, twL);
  __syncthreads();
  // even/odd split: X[k] = E[k] + W^k O[k], E = (Z[k] + conj Z[L-k]) / 2,
  // O = -i (Z[k] - conj Z[L-k]) / 2, and X[L-k] = conj(E - W^k O); X[0] and the Nyquist
  // value X[L] (side plane) from Z[0]
  for (int idx = threadIdx.x; idx < TC * (L / 2 + 1); idx += NT) {
    const int c = idx / (L / 2 + 1), k = idx % (L / 2 + 1);
    const int q = c / R, r = c % R;
    const long long grow = (long long)((T0 << bg.lz) + (r >> bg.ly)) * N + ((T1 << bg.ly) + (r & ((1 << bg.ly) - 1)));
    C* spec = pick(out.spec, q) + (long long)b * spec_len_cx(N);
    C* o = spec + spec_row(N, spec_lzb(N), (int)(grow / N), (int)(grow % N)) * L;
    const C zk = sm[srow(k) * FD::LD + c];
    if (k == 0) {
      o[0] = cmake<C>(zk.x + zk.y, (T)0);
      spec[spec_main_len(N) + grow] = cmake<C>(zk.x - zk.y, (T)0);
      continue;
    }
    const C zm = sm[srow(L - k) * FD::LD + c];
    const T h = (T)0.5;
    const C e = cscale(cadd(zk, cconj(zm)), h);
    const C d = cscale(csub(zk, cconj(zm)), h);
    const C od = cmake<C>(d.y, -d.x);   // -i d
    const C wo = cmul(__ldg(twN + k), od);
    o[k] = cadd(e, wo);
    if (k != L - k) o[L - k] = cconj(csub(e, wo));
  }
}

// Launch shape of the fused deposit for mesh side n (0 rows if n has no fused form).
template <typename T> inline int fused_rows(int n, int nq) {
  switch (n) {
    case 128: return nq == 1 ? FusedDeposit<T, 1, 64>::R : FusedDeposit<T, 4, 64>::R;
    case 256: return nq == 1 ? FusedDeposit<T, 1, 128>::R : FusedDeposit<T, 4, 128>::R;
    case 512: return nq == 1 ? FusedDeposit<T, 1, 256>::R : FusedDeposit<T, 4, 256>::R;
    case 1024: return nq == 1 ? FusedDeposit<T, 1, 512>::R : FusedDeposit<T, 4, 512>::R;
    default: return 0;
  }
}

template <typename T, int NQ, int L>
inline void launch_pull_r2c_L(const BinGeo& bg, int batch, const V4<T>* rec0, const V4<T>* rec1,
                              const unsigned* start, int e_d, const int* e_pi, T mass, const FusedOut<T>& out,
                              const cx_t<T>* tw, cudaStream_t st) {
  using FD = FusedDeposit<T, NQ, L>;
  auto fn = k_pull_r2c<T, NQ, L>;
  if (FD::SMEM > 48 * 1024) ensure_smem_attr((const void*)fn, FD::SMEM);
  fn<<<dim3(bg.ntiles, batch), FD::NT, FD::SMEM, st>>>(bg, rec0, rec1, start, e_d, e_pi, mass, out, tw + L,
                                                        tw + 2 * L);
}

template <typename T, int NQ>
inline int launch_pull_r2c(int n, const BinGeo& bg, int batch, const V4<T>* rec0, const V4<T>* rec1,
                           const unsigned* start, int e_d, const int* e_pi, T mass, const FusedOut<T>& out,
                           const cx_t<T>* tw, cudaStream_t st) {
  switch (n) {
    case 128: launch_pull_r2c_L<T, NQ, 64>(bg, batch, rec0, rec1, start, e_d, e_pi, mass, out, tw, st); break;
    case 256: launch_pull_r2c_L<T, NQ, 128>(bg, batch, rec0, rec1, start, e_d, e_pi, mass, out, tw, st); break;
    case 512: launch_pull_r2c_L<T, NQ, 256>(bg, batch, rec0, rec1, start, e_d, e_pi, mass, out, tw, st); break;
    case 1024: launch_pull_r2c_L<T, NQ, 512>(bg, batch, rec0, rec1, start, e_d, e_pi, mass, out, tw, st); break;
    default: return PM_ERR_ARG;
  }
  return PM_OK;
}

}  // namespace pmgb
