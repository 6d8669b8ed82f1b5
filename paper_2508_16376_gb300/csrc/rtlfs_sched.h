// rtlfs_sched.h -- load-predictor layout and scheduler launchers (rtlfs_sched.cu).
#pragma once
#include "rtlfs_internal.h"

namespace rtlfs {

constexpr int MLP_IN = 5;       // cone size, level, register depth to outputs, width, toggle rate
constexpr int MLP_H = 64;
constexpr int MLP_TILE = 64;    // samples per CTA in the gradient kernel
constexpr int MLP_OFF_B1 = MLP_IN * MLP_H;              // 320
constexpr int MLP_OFF_W2 = MLP_OFF_B1 + MLP_H;          // 384
constexpr int MLP_OFF_B2 = MLP_OFF_W2 + MLP_H * MLP_H;  // 4480
constexpr int MLP_OFF_W3 = MLP_OFF_B2 + MLP_H;          // 4544
constexpr int MLP_OFF_B3 = MLP_OFF_W3 + MLP_H;          // 4608
constexpr int MLP_PARAMS = MLP_OFF_B3 + 1;              // 4609
constexpr uint32_t SORT_BUCKETS = 4096;
// Cycles the toggle-rate feature is measured over: the first min(T, TOGGLE_CYCLES).
constexpr uint32_t TOGGLE_CYCLES = 256;

// Toggle rates are measured over the first min(T, t_limit) cycles of each design.
cudaError_t launch_features(const DevDesign *d_designs, DevFaults f, const float *const *net_static,
                            float *X, float *heur, cudaStream_t s, uint32_t t_limit = TOGGLE_CYCLES);
cudaError_t launch_mlp_forward(const void *wb, const float *X, uint32_t n, float *y, cudaStream_t s);
size_t mlp_grad_smem();
cudaError_t launch_mlp_grad(const void *wb, const float *X, const float *t, uint32_t n, float *grad,
                            float *loss_sum, cudaStream_t s);
cudaError_t launch_mlp_adam(float *master, void *wb, float *grad, float *m, float *v, float lr,
                            float beta1, float beta2, float eps, int step, cudaStream_t s);
// Orders the n faults by descending score into order[]; the first n_heavy become heavy
// items. mm: 2 floats of scratch, hist: SORT_BUCKETS uint32 of scratch. classes = 0: the
// fine order (SORT_BUCKETS score buckets); a power of two up to 64: that many score classes,
// fault-list order kept inside each (cudaErrorInvalidValue otherwise).
cudaError_t launch_order(const float *score, uint32_t n, float *mm, uint32_t *hist, uint32_t *order,
                         uint32_t n_heavy, HeavyItem *items, cudaStream_t s, uint32_t classes = 0);

}  // namespace rtlfs
