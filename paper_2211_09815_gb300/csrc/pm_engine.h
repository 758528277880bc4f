// Precision-independent interface of the PM engine behind the C ABI.
#pragma once
#include <cuda_runtime.h>

#include "../../include/pm.h"

namespace pmgb {

struct EngineBase {
  virtual ~EngineBase() {}
  virtual int forward(void* disp, void* mom, void* dens) = 0;
  virtual int loss_mse(const void* target, double* loss, void* djdd) = 0;
  virtual int adjoint(const void* djdd, const void* djdx, const void* djdp, void* djdw, double* djdth) = 0;
  virtual int op_density(const void* disp, void* dens) = 0;
  virtual int op_force(const void* disp, const void* pi, void* acc, void* alpha) = 0;
  virtual int op_fft(int dir, const void* in, void* out) = 0;
  virtual int op_za(void* s1) = 0;
  virtual int op_ic(void* s0, void* p0) = 0;
  virtual int set_snapshots(int ns, const int* steps, void* disp, void* dens, const void* gdisp,
                            const void* gdens) = 0;
  virtual int set_snapshot_momenta(void* mom, const void* gmom) = 0;
  virtual int set_interp_snapshots(int na, const double* a, void* disp, void* dens, const void* gdisp,
                                   const void* gdens) = 0;
  virtual int get_fixed_state(long long* u, long long* w) = 0;
  virtual long long scratch_bytes() const = 0;
  virtual int profile(int enable) = 0;
  virtual int profile_read(double* ms, long long* launches) = 0;
  virtual int set_inputs(const double* theta, const void* omega) = 0;
  virtual int gradient_graph(const void* target, double* loss, void* gw, double* gt) = 0;
  virtual int power_spectrum(const void* dens, double* pk, double* kmean, double* nmodes) = 0;
  virtual int loss_power(const void* dens, const double* tgt, const double* w, double* loss, void* djdd) = 0;
  virtual int gradient(const void* omega, const void* target, double* loss, void* grad_omega, double* grad_theta) = 0;
  virtual int get_tuning(pm_tuning* t) = 0;
  virtual int set_tuning(const pm_tuning* t) = 0;
  virtual int autotune(int reps, pm_tuning* chosen, double* ms_best) = 0;
  // synchronise the stream; PM_ERR_TIMEOUT if a bounded device wait gave up since the
  // last check (the flag is cleared)
  virtual int check() = 0;
  // test hook: spin limit of the first mbarrier wait of every TMA-staged CTA (< 0: normal)
  virtual void set_first_wait(int spins) = 0;
};

// Creates the engine for cfg->precision; returns a status and sets *out on success.
int make_engine(const pm_config* cfg, const double* theta, const void* omega, cudaStream_t st, EngineBase** out);

// Record the last CUDA error message for pm_last_cuda_error.
void set_cuda_error(cudaError_t e);

// Host-side fault injection for the allocation path (pm_debug_fail_alloc): false when the
// next device allocation is to fail.  Bytes held by all engines (pm_debug_live_bytes).
bool alloc_gate();
void live_bytes_add(long long delta);

}  // namespace pmgb
