// internal.h -- declarations shared by the library's translation units.
// Not part of the public ABI (include/fx.h is).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "../../include/fx.h"

namespace fxi {

constexpr int kPols = 2;

// Handle state. Device pointers are owned by the handle.
struct Handle {
    fx_params p;                 // copy; host pointers inside are cleared
    int I, I_pad, S_pad, B;
    float operand_scale;
    int device;
    // device buffers
    float *d_taps = nullptr;           // [T*C]
    float2 *d_twiddle = nullptr;       // [C]  exp(-2 pi i m / C), from host FP64
    double *d_centres = nullptr;       // [SB]
    float2 *d_phase = nullptr;         // [SB][N][C] (phi0 mod 2pi, per-spectrum step)
    int *d_status = nullptr;           // device-side error word
    int2 *d_xf32_tiles = nullptr;      // tile list of the FP32 correlator
    int xf32_ntiles = 0;
    int xf32_mode = 1;                 // its form: 0 2x4 tiles, 1 4x4 tiles, 2 2x4 tiles with 3 multiplications
    double *d_adj_partial = nullptr;   // [adjoint CTAs][I][4] per-CTA gradient sums
    // streaming (FX_FLAG_STREAMING): FIR history ping-pong + assembled block
    int hist_len = 0;                  // samples of history per (subband, station)
    void *d_hist[2] = {nullptr, nullptr};
    int hist_cur = 0;
    void *d_block = nullptr;
    // fx_channelize_correlate (chunk_spectra > 0): two operand buffers of one piece
    void *d_chunk[2] = {nullptr, nullptr};
    // beamformer (max_beams > 0): weight table [SB][C][re/im][ceil64(max_beams)][64]
    unsigned short *d_bfw = nullptr;
    // host pipeline (fx_process_host), when host_chunk_subbands > 0
    struct HostPipe *pipe = nullptr;
    int num_sms = 0;
    long long tc_timeout_cycles = 0;   // budget of every bounded device-side wait
    int tc_test_no_tma = 0;            // failure-detection test hook (FX_FLAG_TEST_NO_LOADS)
};

// ppf.cu
cudaError_t launch_ppf(const Handle &h, const void *raw, float2 *chan, cudaStream_t st);
bool ppf_supported(int C, int T);

// channelize_correct_impl.cuh (flags: [N][S] lost-data weights or null). A window
// produces spectra [s_base, s_end) (s_base a multiple of 16) into an output
// whose spectrum stride is s_out (spectrum s at s - s_base); null = the block.
struct FWindow {
    int s_base, s_end, s_out;
};
cudaError_t launch_channelize_correct(const Handle &h, const void *raw, const float *bandpass, const float2 *gains,
                                      void *corr, cudaStream_t st, const float *flags = nullptr,
                                      const FWindow *window = nullptr);

// stream.cu
int raw_sample_bytes(const Handle &h);   // bytes of one time sample of one station (both pols)
cudaError_t launch_stream_assemble(const Handle &h, const void *d_new, const int *shift, cudaStream_t st);
cudaError_t launch_stream_history(Handle &h, const void *d_new, cudaStream_t st);
cudaError_t launch_baseline_counts(const Handle &h, const float *flags, float *counts, cudaStream_t st);

// correct.cu
cudaError_t launch_phase_table(const Handle &h, const double *tau_b, const double *tau_e,
                               cudaStream_t st);
cudaError_t launch_correct(const Handle &h, const float2 *chan, const float *bandpass,
                           const float2 *gains, void *corr, cudaStream_t st);
constexpr int kMaxDevices = 64;
cudaError_t launch_correct_f32_noalloc(int N, int SB, int C, int S, double fs, const double *centres,
                                       const double *tau_b, const double *tau_e, const float *bandpass,
                                       const float2 *gains, const float2 *chan, float2 *corr, cudaStream_t st);

// xcorr_f32.cu
int xf32_build_tiles(int N, int RS, int2 *host_tiles /* may be null: count only */);
cudaError_t launch_xcorr_f32(const Handle &h, const float2 *corr, float2 *vis, cudaStream_t st,
                             bool accumulate = false);   // accumulate: add to vis

// host_pipeline.cu
cudaError_t pipe_create(Handle &h, int chunk);
void pipe_destroy(Handle &h);
cudaError_t pipe_run(Handle &h, const void *h_raw, const double *h_tb, const double *h_te, const float *h_bp,
                     const float *h_gains, float *h_vis, cudaStream_t st);

// adjoint.cu
int adjoint_blocks(const Handle &h);
cudaError_t launch_apply_gains(const Handle &h, const float2 *R, const float2 *gains, const double *tau,
                               float2 *V, cudaStream_t st);
cudaError_t launch_adjoint(const Handle &h, const float2 *R, const float2 *G, const float2 *gains,
                           const double *tau, float2 *grad_gains, double *grad_tau, cudaStream_t st);
cudaError_t launch_weight_spectra(const Handle &h, void *corr, cudaStream_t st);
cudaError_t launch_adjoint_interp(const Handle &h, const float2 *K, const float2 *M1, const float2 *G,
                                  const float2 *gains, float2 *grad_gains, double *grad_tb, double *grad_te,
                                  cudaStream_t st);

// beamform.cu
size_t bf_weight_bytes(const Handle &h, int n_beams);
cudaError_t launch_beamform_incoherent(const Handle &h, const void *corr, const float *weights, int mode, int tint,
                                       float *out, cudaStream_t st);
cudaError_t launch_beamform(const Handle &h, const void *corr, int n_beams, const double *delays,
                            const float *weights, int mode, int tint, float *out, cudaStream_t st);

// xcorr_tf32.cu (FX_TF32_SPLIT)
bool xtf32_supported(int I_pad, int S_pad);
cudaError_t launch_xcorr_tf32(const Handle &h, const float *corr, float2 *vis, cudaStream_t st,
                             bool accumulate = false);    // accumulate: add to vis

// probe.cu
cudaError_t launch_ffma_probe(int iterations, int blocks, float *sink, cudaStream_t st);

// fx_api.cu: the X-stage of the handle's precision
bool xstage_supported(const Handle &h);
cudaError_t launch_xstage(const Handle &h, const void *corr, float2 *vis, cudaStream_t st, bool accumulate = false);

// xcorr_tc.cu
bool xtc_plan(const Handle &h, int *rload, int *stages, unsigned *stage_bytes);
cudaError_t launch_xcorr_tc(const Handle &h, const void *corr, float2 *vis, cudaStream_t st,
                            bool accumulate = false);    // accumulate: add to vis

}  // namespace fxi

// batched tensor-core X-stage (xcorr_tc.cu)
cudaError_t fxi_batch_create(const fx_job *jobs, int n_jobs, int precision, float scale, int num_sms,
                             fx_batch **out, const char **why);
cudaError_t fxi_batch_launch(fx_batch *b, cudaStream_t st);
cudaError_t fxi_batch_autotune(fx_batch *b, int reps, cudaStream_t st);
void fxi_batch_destroy(fx_batch *b);
const char *fxi_batch_describe(const fx_batch *b);
int *fxi_batch_status(fx_batch *b);
int fxi_batch_device(const fx_batch *b);
