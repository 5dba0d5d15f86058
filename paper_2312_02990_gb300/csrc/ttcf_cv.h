// ttcf_cv.h -- declarations of the control-variate kernels (ttcf_cv.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ttcf_internal.h"

namespace ttcf {

constexpr int CV_NF = 32;    // features
constexpr int CV_H = 128;    // hidden units per layer
constexpr int CV_NP = CV_H * CV_NF + CV_H + CV_H * CV_H + CV_H + CV_H + 1;   // 20865

struct CvFeatArgs {
    const double *raw;      // [G][FEAT_RAW] from the features kernel
    const double *alpha;    // [G] mother alpha, or null
    int reset_alpha;
    int M;
    int maps[4];
    long long D;
    int N;
    double V;
    float *X;               // [D][CV_NF] out
};

cudaError_t cv_launch_features(const CvFeatArgs &a, cudaStream_t st);

// Raw features (FEAT_RAW doubles per state, the layout of FEAT_RAW) of G
// phase points of one bulk system, in FP32 arithmetic with
// FP64 block sums: kinetic sums, WCA virial and energy, sum p^2, slab modes.
// src holds [G][6][N] values: IEEE doubles (kind 0) or float-pair slots
// (kind 1, hi part used); both give the same FP32 inputs.
struct CvRawArgs {
    const void *src;
    int kind;
    int N, G;
    int nc[3], ncell;       // cells of width >= r_c
    double L[3];
    double *raw;            // [G][FEAT_RAW] out
};
cudaError_t cv_launch_raw_features(const CvRawArgs &a, cudaStream_t st);
size_t cv_raw_smem_bytes(int N, int ncell);
cudaError_t cv_launch_targets(const double *B, const double *Omega, const double *gamma, int M,
                              long long D, int S, double ds, double *z, cudaStream_t st);
cudaError_t cv_launch_colstats(const float *A, int ld, const int *rows, int n, int ncols,
                               double *stats, cudaStream_t st);
cudaError_t cv_launch_standardize(float *X, long long n, const double *stats, float *y,
                                  const double *zstats, const double *z, cudaStream_t st);
cudaError_t cv_launch_predict(const __nv_bfloat16 *wb, const float *X, long long n, float *out,
                              int nsm, cudaStream_t st);
// The tensor-core forward pass records a timed-out wait in a device flag:
// cleared by cv_tc_reset, read (with a stream synchronisation) by cv_tc_failed.
cudaError_t cv_tc_reset(cudaStream_t st);
cudaError_t cv_tc_failed(cudaStream_t st, int *failed);
cudaError_t cv_launch_grad(const __nv_bfloat16 *wb, const float *X, const float *y, const int *idx,
                           long long base, int nbatch, float *part, double *lpart, int *step,
                           cudaStream_t st);
cudaError_t cv_launch_adam(const float *part, int ntiles, const double *lpart, float *grad, double *loss,
                           float *w, float *m, float *v, __nv_bfloat16 *wb, const int *step, float lr,
                           float b1, float b2, float eps, cudaStream_t st);
cudaError_t cv_launch_to_bf16(const float *w, __nv_bfloat16 *wb, cudaStream_t st);
cudaError_t cv_launch_group(const double *z, const float *f, const double *zstats, int M,
                            const int *groups, int ng, double *yg, double *hg, cudaStream_t st);
cudaError_t cv_launch_estimate(const double *yD, const double *hD, int nD, const double *hM, int nM,
                               int fit_c, double c_in, double *out, cudaStream_t st);
size_t mlp_smem_bytes();

}  // namespace ttcf
