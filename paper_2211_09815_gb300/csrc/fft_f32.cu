// Explicit float instantiations of the FFT passes.
#include "fft_impl.cuh"

namespace pmgb {
template int fft_cols<float>(int, int, const SeqMap&, const SeqMap&, const ColBufs<float>&, int, const cx_t<float>*,
                             cudaStream_t);
template int fft_x_r2c<float>(int, const RowJob<float>&, int, int, const cx_t<float>*, cudaStream_t);
template int fft_x_c2r<float>(int, const RowJob<float>&, int, int, const cx_t<float>*, cudaStream_t);
template int fft_fused_z<float>(int, const ZJob<float>&, bool, const cx_t<float>*, cudaStream_t);
template int fft_cols_tma<float>(int, int, int, int, const CUtensorMap*, cx_t<float>* const*, int, const cx_t<float>*,
                                const WaitCtl&, int, cudaStream_t);
template int fft_fused_tma<float>(int, bool, const CUtensorMap*, const CUtensorMap*, const ZJob<float>&, const cx_t<float>*, const WaitCtl&, int,
                                 cudaStream_t);
template int fft_fused_side<float>(int, const ZJob<float>&, bool, const cx_t<float>*, cudaStream_t);
template int make_spec_tensor_maps<float>(int, int, cx_t<float>*, CUtensorMap*, CUtensorMap*);
template int fft_x_c2r4<float>(int, const RowJob<float>&, int, int, void*, signed char*, const cx_t<float>*, cudaStream_t);
template int fft_cols_split<float>(int, const SeqMap&, const SeqMap&, cx_t<float>*, cx_t<float>*, const cx_t<float>*,
                                   cudaStream_t);
template int fft_cols_merge<float>(int, const SeqMap&, const SeqMap&, cx_t<float>*, cx_t<float>*, const cx_t<float>*,
                                   cudaStream_t);
template int fft_ysplit_tma<float>(int, int, const CUtensorMap*, cx_t<float>*, cx_t<float>*, const cx_t<float>*, const WaitCtl&, int,
                                   cudaStream_t);
template int fft_ymerge_tma<float>(int, int, const CUtensorMap*, cx_t<float>*, const cx_t<float>*, const WaitCtl&, int, cudaStream_t);
}  // namespace pmgb
