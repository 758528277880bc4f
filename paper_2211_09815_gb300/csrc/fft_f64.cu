// Explicit double instantiations of the FFT passes.
#include "fft_impl.cuh"

namespace pmgb {
template int fft_cols<double>(int, int, const SeqMap&, const SeqMap&, const ColBufs<double>&, int, const cx_t<double>*,
                             cudaStream_t);
template int fft_x_r2c<double>(int, const RowJob<double>&, int, int, const cx_t<double>*, cudaStream_t);
template int fft_x_c2r<double>(int, const RowJob<double>&, int, int, const cx_t<double>*, cudaStream_t);
template int fft_fused_z<double>(int, const ZJob<double>&, bool, const cx_t<double>*, cudaStream_t);
template int fft_cols_tma<double>(int, int, int, int, const CUtensorMap*, cx_t<double>* const*, int, const cx_t<double>*,
                                const WaitCtl&, int, cudaStream_t);
template int fft_fused_tma<double>(int, bool, const CUtensorMap*, const CUtensorMap*, const ZJob<double>&, const cx_t<double>*, const WaitCtl&, int,
                                 cudaStream_t);
template int fft_fused_side<double>(int, const ZJob<double>&, bool, const cx_t<double>*, cudaStream_t);
template int make_spec_tensor_maps<double>(int, int, cx_t<double>*, CUtensorMap*, CUtensorMap*);
template int fft_x_c2r4<double>(int, const RowJob<double>&, int, int, void*, signed char*, const cx_t<double>*, cudaStream_t);
template int fft_cols_split<double>(int, const SeqMap&, const SeqMap&, cx_t<double>*, cx_t<double>*, const cx_t<double>*,
                                   cudaStream_t);
template int fft_cols_merge<double>(int, const SeqMap&, const SeqMap&, cx_t<double>*, cx_t<double>*, const cx_t<double>*,
                                   cudaStream_t);
template int fft_ysplit_tma<double>(int, int, const CUtensorMap*, cx_t<double>*, cx_t<double>*, const cx_t<double>*, const WaitCtl&, int,
                                   cudaStream_t);
template int fft_ymerge_tma<double>(int, int, const CUtensorMap*, cx_t<double>*, const cx_t<double>*, const WaitCtl&, int, cudaStream_t);
}  // namespace pmgb
