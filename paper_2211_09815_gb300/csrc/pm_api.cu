// C ABI of libpmgb (declared in include/pm.h): host-side validation, context lifetime
// and dispatch to the precision-specific engine.
#include <atomic>
#include <cmath>
#include <mutex>
#include <set>
#include <string>
#include <utility>

#include "pm_engine.h"
#include "pm_internal.h"

namespace pmgb {

template <typename T>
int make_engine_t(const pm_config* cfg, const double* theta, const void* omega, cudaStream_t st, EngineBase** out);

static thread_local std::string g_cuda_err;

void set_cuda_error(cudaError_t e) { g_cuda_err = cudaGetErrorString(e); }

void ensure_smem_attr(const void* fn, int bytes) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({dev, fn})) return;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  done.insert({dev, fn});
}

static std::mutex g_hook_mu;
static long long g_fail_after = -1;             // allocations still allowed (-1: no failure)
static std::atomic<long long> g_live_bytes{0};

bool alloc_gate() {
  std::lock_guard<std::mutex> lk(g_hook_mu);
  if (g_fail_after < 0) return true;
  if (g_fail_after == 0) {
    g_fail_after = -1;
    return false;
  }
  --g_fail_after;
  return true;
}
void live_bytes_add(long long delta) { g_live_bytes += delta; }

static bool pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

static int validate(const pm_config* c, const double* theta) {
  if (!c || !theta) return PM_ERR_ARG;
  if (!(c->box > 0) || !std::isfinite(c->box)) return PM_ERR_ARG;
  if (!pow2(c->n_mesh) || !pow2(c->n_ptcl) || c->n_ptcl < 4 || c->n_mesh < 8 || c->n_mesh > 1024) return PM_ERR_ARG;
  if (c->n_mesh % c->n_ptcl != 0) return PM_ERR_ARG;
  if (c->n_steps < 1 || c->batch < 1 || c->ckpt_every < 0) return PM_ERR_ARG;
  if (c->lpt_order < 0 || c->lpt_order > 2) return PM_ERR_ARG;
  if (c->fixed_state < 0 || c->fixed_state > 1 || (c->fixed_state && c->ckpt_every > 0)) return PM_ERR_ARG;
  if (c->half_force < 0 || c->half_force > 1 || (c->half_force && c->precision != PM_F32)) return PM_ERR_ARG;
  if (!(c->a0 > 0) || !(c->a1 > c->a0) || !std::isfinite(c->a1)) return PM_ERR_ARG;
  if (c->precision != PM_F32 && c->precision != PM_F64) return PM_ERR_ARG;
  if ((long long)c->batch * c->n_mesh * c->n_mesh * (c->n_mesh / 2) >= (1LL << 31)) return PM_ERR_ARG;
  for (int b = 0; b < c->batch; ++b)
    for (int j = 0; j < 5; ++j)
      if (!std::isfinite(theta[5 * b + j])) return PM_ERR_NONFINITE;
  for (int b = 0; b < c->batch; ++b) {
    const double* t = theta + 5 * b;
    if (!(t[0] > 0) || !(t[2] > 0) || !(t[2] <= 1) || !(t[3] >= 0) || !(t[3] < t[2]) || !(t[4] > 0)) return PM_ERR_ARG;
  }
  return PM_OK;
}

}  // namespace pmgb

using namespace pmgb;

struct pm_ctx {
  EngineBase* eng;
  pm_config cfg;
};

extern "C" {

int pm_init(pm_ctx** out, const pm_config* cfg, const double* theta, const void* omega, void* stream) {
  if (!out || !omega) return PM_ERR_ARG;
  const int v = validate(cfg, theta);
  if (v != PM_OK) return v;
  EngineBase* e = nullptr;
  int r;
  try {
    r = cfg->precision == PM_F32 ? make_engine_t<float>(cfg, theta, omega, (cudaStream_t)stream, &e)
                                 : make_engine_t<double>(cfg, theta, omega, (cudaStream_t)stream, &e);
  } catch (...) {
    return PM_ERR_OOM;
  }
  if (r != PM_OK) return r;
  *out = new pm_ctx{e, *cfg};
  return PM_OK;
}

int pm_forward(pm_ctx* ctx, void* disp_out, void* mom_out, void* dens_out) {
  if (!ctx) return PM_ERR_ARG;
  return ctx->eng->forward(disp_out, mom_out, dens_out);
}

int pm_loss_mse(pm_ctx* ctx, const void* target, double* loss_out, void* dJ_ddens_out) {
  if (!ctx || !target || !dJ_ddens_out) return PM_ERR_ARG;
  return ctx->eng->loss_mse(target, loss_out, dJ_ddens_out);
}

int pm_adjoint(pm_ctx* ctx, const void* dJ_ddens, const void* dJ_ddisp, const void* dJ_dmom, void* dJ_domega,
               double* dJ_dtheta) {
  if (!ctx) return PM_ERR_ARG;
  return ctx->eng->adjoint(dJ_ddens, dJ_ddisp, dJ_dmom, dJ_domega, dJ_dtheta);
}

int pm_set_inputs(pm_ctx* ctx, const double* theta, const void* omega) {
  if (!ctx) return PM_ERR_ARG;
  if (theta) {
    pm_config c = ctx->cfg;
    const int v = validate(&c, theta);
    if (v != PM_OK) return v;
  }
  return ctx->eng->set_inputs(theta, omega);
}

int pm_gradient(pm_ctx* ctx, const void* omega, const void* target, double* loss, void* grad_omega,
                double* grad_theta) {
  if (!ctx || !target) return PM_ERR_ARG;
  return ctx->eng->gradient(omega, target, loss, grad_omega, grad_theta);
}

int pm_gradient_graph(pm_ctx* ctx, const void* target, double* loss, void* grad_omega, double* grad_theta) {
  if (!ctx || !target) return PM_ERR_ARG;
  return ctx->eng->gradient_graph(target, loss, grad_omega, grad_theta);
}

int pm_power_spectrum(pm_ctx* ctx, const void* dens, double* pk, double* kmean, double* nmodes) {
  if (!ctx || !pk) return PM_ERR_ARG;
  return ctx->eng->power_spectrum(dens, pk, kmean, nmodes);
}

int pm_loss_power(pm_ctx* ctx, const void* dens, const double* pk_target, const double* weights, double* loss_out,
                  void* dJ_ddens_out) {
  if (!ctx || !pk_target || !weights || !dJ_ddens_out) return PM_ERR_ARG;
  return ctx->eng->loss_power(dens, pk_target, weights, loss_out, dJ_ddens_out);
}

int pm_profile(pm_ctx* ctx, int enable) {
  if (!ctx) return PM_ERR_ARG;
  return ctx->eng->profile(enable);
}

int pm_profile_read(pm_ctx* ctx, double* ms, long long* launches) {
  if (!ctx) return PM_ERR_ARG;
  return ctx->eng->profile_read(ms, launches);
}

int pm_destroy(pm_ctx* ctx) {
  if (!ctx) return PM_ERR_ARG;
  delete ctx->eng;
  delete ctx;
  return PM_OK;
}

const char* pm_status_string(int s) {
  switch (s) {
    case PM_OK: return "ok";
    case PM_ERR_ARG: return "invalid argument";
    case PM_ERR_OOM: return "device allocation failed";
    case PM_ERR_CUDA: return "CUDA error";
    case PM_ERR_NONFINITE: return "non-finite input";
    case PM_ERR_OVERFLOW: return "fixed-point range exceeded";
    case PM_ERR_TIMEOUT: return "bounded device wait gave up";
    case PM_ERR_STATE: return "call out of order";
    default: return "unknown status";
  }
}

const char* pm_last_cuda_error(void) { return g_cuda_err.c_str(); }

long long pm_scratch_bytes(const pm_ctx* ctx) { return ctx ? ctx->eng->scratch_bytes() : 0; }

int pm_get_tuning(pm_ctx* ctx, pm_tuning* out) {
  if (!ctx || !out) return PM_ERR_ARG;
  return ctx->eng->get_tuning(out);
}

int pm_set_tuning(pm_ctx* ctx, const pm_tuning* t) {
  if (!ctx || !t) return PM_ERR_ARG;
  return ctx->eng->set_tuning(t);
}

int pm_autotune(pm_ctx* ctx, int reps, pm_tuning* chosen, double* ms_best) {
  if (!ctx || reps < 0 || reps > 100) return PM_ERR_ARG;
  return ctx->eng->autotune(reps, chosen, ms_best);
}

int pm_op_density(pm_ctx* ctx, const void* disp, void* dens_out) {
  if (!ctx || !disp || !dens_out) return PM_ERR_ARG;
  return ctx->eng->op_density(disp, dens_out);
}

int pm_op_force(pm_ctx* ctx, const void* disp, void* acc_out) {
  if (!ctx || !disp || !acc_out) return PM_ERR_ARG;
  return ctx->eng->op_force(disp, nullptr, acc_out, nullptr);
}

int pm_op_force_vjp(pm_ctx* ctx, const void* disp, const void* pi, void* acc_out, void* alpha_out) {
  if (!ctx || !disp || !pi || !acc_out || !alpha_out) return PM_ERR_ARG;
  return ctx->eng->op_force(disp, pi, acc_out, alpha_out);
}

int pm_op_fft(pm_ctx* ctx, int dir, const void* in, void* out) {
  if (!ctx || !in || !out || (dir != -1 && dir != 1)) return PM_ERR_ARG;
  return ctx->eng->op_fft(dir, in, out);
}

int pm_op_za(pm_ctx* ctx, void* s1_out) {
  if (!ctx || !s1_out) return PM_ERR_ARG;
  return ctx->eng->op_za(s1_out);
}

int pm_set_snapshots(pm_ctx* ctx, int nsnap, const int* steps, void* disp_out, void* dens_out,
                     const void* dJ_ddisp, const void* dJ_ddens) {
  if (!ctx) return PM_ERR_ARG;
  return ctx->eng->set_snapshots(nsnap, steps, disp_out, dens_out, dJ_ddisp, dJ_ddens);
}

int pm_set_snapshot_momenta(pm_ctx* ctx, void* mom_out, const void* dJ_dmom) {
  if (!ctx) return PM_ERR_ARG;
  return ctx->eng->set_snapshot_momenta(mom_out, dJ_dmom);
}

int pm_set_interp_snapshots(pm_ctx* ctx, int na, const double* a, void* disp_out, void* dens_out,
                            const void* dJ_ddisp, const void* dJ_ddens) {
  if (!ctx) return PM_ERR_ARG;
  return ctx->eng->set_interp_snapshots(na, a, disp_out, dens_out, dJ_ddisp, dJ_ddens);
}

int pm_get_fixed_state(pm_ctx* ctx, long long* disp_fixed, long long* mom_fixed) {
  if (!ctx) return PM_ERR_ARG;
  return ctx->eng->get_fixed_state(disp_fixed, mom_fixed);
}

int pm_op_ic(pm_ctx* ctx, void* s0_out, void* p0_out) {
  if (!ctx) return PM_ERR_ARG;
  return ctx->eng->op_ic(s0_out, p0_out);
}

int pm_check(pm_ctx* ctx) {
  if (!ctx) return PM_ERR_ARG;
  return ctx->eng->check();
}

int pm_debug_fail_alloc(long long after) {
  std::lock_guard<std::mutex> lk(g_hook_mu);
  g_fail_after = after < 0 ? -1 : after;
  return PM_OK;
}

long long pm_debug_live_bytes(void) { return g_live_bytes.load(); }

int pm_debug_first_wait(pm_ctx* ctx, int spins) {
  if (!ctx) return PM_ERR_ARG;
  ctx->eng->set_first_wait(spins);
  return PM_OK;
}

}  // extern "C"

namespace pmgb {

bool tma_supported(int n) { return n == 128 || n == 256 || n == 512 || n == 1024; }

}  // namespace pmgb
