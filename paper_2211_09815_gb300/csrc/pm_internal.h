// Internal declarations shared by the CUDA translation units of libpmgb.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pm.h"
#include "common.cuh"

namespace pmgb {

// Address map of a batch of length-L sequences for a column FFT pass.  Sequence s,
// element r lives at  o1*os1 + o0*os0 + col*cs + r*es  (complex elements) with
// col = s % ncols, o0 = (s / ncols) % n0, o1 = s / (ncols * n0).
struct SeqMap {
  long long es, cs;
  int ncols;
  long long os0;
  int n0;
  long long os1;
  int nseq;
};

template <typename T> struct ColBufs { cx_t<T>* p[4]; };

// One buffer of a row (x) pass.  R2C: real -> spec.  C2R: spec -> real.
template <typename T> struct RowBuf {
  void* real;           // real mesh (T)
  long long real_is;    // instance stride of `real` in elements
  cx_t<T>* spec;        // spectrum buffer (main + side)
};
template <typename T> struct RowJob {
  RowBuf<T> b[4];
  int lzb;              // log2 of the z blocking of the spectra's main rows (spec_row); 0: plain
};

// Fused z pass with the Green's function G = coef[b] / n^2 * (deconvolution) per mode.
// Force: in[0] = delta^ -> out[0] = z force (-i k_0 G), out[1] = U (G, shared by the y and
// x forces).  Adjoint: in[0] = P_0, in[1] = V -> out[0] = psi.
template <typename T> struct ZJob {
  cx_t<T>* in[3];
  cx_t<T>* out[3];
  const T* coef;    // [batch]
  const T* dtab;    // [n] 1/sinc^4(pi f/n) or null
  int batch;
};

template <typename T>
int fft_cols(int n, int dir, const SeqMap& mm, const SeqMap& ms, const ColBufs<T>& bufs, int nbuf,
             const cx_t<T>* tw, cudaStream_t st);
// y passes of the separable force components (main columns of mm and side columns of ms):
// split (inverse): out1 = IFFT(u), u = IFFT(-i k_1 u); merge (forward):
// p1 = i (k_1 FFT(p1) + k_2 FFT(p2))
template <typename T>
int fft_cols_split(int n, const SeqMap& mm, const SeqMap& ms, cx_t<T>* u, cx_t<T>* out1, const cx_t<T>* tw,
                   cudaStream_t st);
template <typename T>
int fft_cols_merge(int n, const SeqMap& mm, const SeqMap& ms, cx_t<T>* p1, cx_t<T>* p2, const cx_t<T>* tw,
                   cudaStream_t st);
template <typename T>
int fft_x_r2c(int n, const RowJob<T>& job, int nbuf, int nrows, const cx_t<T>* tw,
              cudaStream_t st);
template <typename T>
int fft_x_c2r(int n, const RowJob<T>& job, int nbuf, int nrows, const cx_t<T>* tw, cudaStream_t st);
// C2R of up to four components into one interleaved [cell][4] real mesh; component dq
// (none if dq < 0) is multiplied by -i k_x first
template <typename T>
int fft_x_c2r4(int n, const RowJob<T>& job, int nrows, int dq, void* out, signed char* fexp, const cx_t<T>* tw,
               cudaStream_t st);
template <typename T>
int fft_fused_z(int n, const ZJob<T>& job, bool adjoint, const cx_t<T>* tw, cudaStream_t st);

// Bounded mbarrier waits of the TMA-staged passes: the device flag a wait that gives up
// sets, and the spin limit of each CTA's first wait (negative: the normal limit; a test
// hook sets 0 so that the first wait gives up at once).
struct WaitCtl {
  int* err;
  int first_wait;
};

// TMA-staged persistent column passes over the main half spectrum (mesh sizes 128..1024).
bool tma_supported(int n);
template <typename T>
int fft_cols_tma(int n, int batch, int dir, int zaxis, const CUtensorMap* maps, cx_t<T>* const* bufs, int nb,
                 const cx_t<T>* tw, const WaitCtl& wc, int nsm, cudaStream_t st);
template <typename T>
int fft_fused_tma(int n, bool adjoint, const CUtensorMap* maps, const CUtensorMap* omaps, const ZJob<T>& job,
                  const cx_t<T>* tw, const WaitCtl& wc, int nsm, cudaStream_t st);
// the same split and merge over the main spectrum with TMA-staged tiles
template <typename T>
// umaps: y maps of u and out1
int fft_ysplit_tma(int n, int batch, const CUtensorMap* umaps, cx_t<T>* u, cx_t<T>* out1, const cx_t<T>* tw,
                   const WaitCtl& wc, int nsm, cudaStream_t st);
template <typename T>
int fft_ymerge_tma(int n, int batch, const CUtensorMap* pmaps, cx_t<T>* p1, const cx_t<T>* tw, const WaitCtl& wc, int nsm,
                   cudaStream_t st);
// the side-plane (kx = n/2) tiles of the fused z passes only
template <typename T>
int fft_fused_side(int n, const ZJob<T>& job, bool adjoint, const cx_t<T>* tw, cudaStream_t st);
// tensor maps of one spectrum buffer for the y pass (box along y) and the z pass (box along z)
template <typename T>
int make_spec_tensor_maps(int n, int batch, cx_t<T>* buf, CUtensorMap* ymap, CUtensorMap* zmap);

// Set the dynamic shared-memory limit of a kernel once per device.
void ensure_smem_attr(const void* fn, int bytes);

}  // namespace pmgb
