// Internal declarations shared by the library's translation units: the plan object,
// the launchers of the setup kernels (Alg. 1) and of the solve passes (Alg. 2).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

#include "../../include/superpot.h"
#include "sp_common.cuh"
#include "sp_df32.cuh"

struct sp_plan_s {
    int n[3];        // grid points per axis
    int N[3];        // padded FFT lengths 2n
    double lo[3], hi[3];
    double h[3];     // grid spacing (hi - lo)/(n - 1)
    double L[3];     // window half-width n h
    sp_precision prec;
    int max_batch;
    int ldz;         // row stride (in complex elements) of the kz dimension, >= n2 + 1
    long long plane; // complex elements per x-plane of the workspace: 2 n1 ldz
    // GS table (eq. sin_1_x)
    double eps, delta, h_tau, eta;
    int gs_terms;    // S + 1 (0 until known)
    bool gs_user;
    double* d_gs_w;
    double* d_gs_a;
    int gs_cap;      // allocated length of d_gs_w / d_gs_a
    double* h_gs_a;  // host copy of the exponents (decides the full-line rows)
    // 1D integral tables per axis [s][k], kept for diagnostics; axes with equal
    // (n, L) share the table of the first such axis
    double* d_G[3];
    double* d_H[3];
    // multiplier octant [|k1|][|k0|][kz] with row stride ldz, scaled by 1/Ntilde
    double* d_M64;
    float* d_M32;
    df32* d_Mdf;     // double-float copy (SP_DF32 plans)
    // twiddles exp(-2 pi i j / N_p), j < N_p, per axis (FP64 and FP32)
    cpx<double>* d_tw64[3];
    cpx<float>* d_tw32[3];
    cpx<df32>* d_twdf[3];
    RadixPlan rp[3];
    // Bluestein axes (2n with a prime factor above 7; rp[ax].nst == 0 there): the circular
    // convolution length M (a power of two >= 4n - 1), its radix plan, and the device table
    // [chirp, 2n][filter spectrum, forward, M][filter spectrum, inverse, M][twiddles, M]
    // of complex values in the plan's arithmetic type; NULL on the other axes
    int blue_M[3];
    RadixPlan blue_rp[3];
    void* d_blue[3];
    // solve workspace: max_batch x n0 x 2n1 x ldz complex (pass precision)
    void* d_work;
    size_t work_bytes;
    bool ready;
    int device;
    int kernel;      // sp_kernel
    // the plan's last recorded work: every entry point that issues work on a stream records
    // this event after it, so destroy and sp_plan_sync wait for the plan alone
    cudaEvent_t done;
    bool done_recorded;
    // device status word: set by a kernel whose bounded wait gave up (SP_ERR_TIMEOUT),
    // read and cleared by sp_plan_sync
    int* d_status;
    // device memory of the plan: every allocation, released in reverse order at destroy,
    // through the caller's allocator when one was given, else cudaFree
    sp_allocator alloc;
    bool has_alloc;
    // without a caller's allocator: stream-ordered allocations (cudaMallocAsync) on this
    // private stream, freed there (cudaFreeAsync) after the plan's last work, so that
    // destroy never waits for the device
    cudaStream_t mem_st;
    int nalloc;
    void* alloc_ptr[32];
    size_t alloc_bytes[32];
    // sp_solve_host staging (created by its first call): two input and two output device
    // buffers, a host-to-device and a device-to-host copy stream, and their events
    void* d_stage[4];
    cudaStream_t copy_st[2];
    cudaEvent_t stage_ev[6];  // loaded[2], solved[2], fetched[2]
    bool staged;
    // tiles of the register-resident passes (0 = built-in default): columns per CTA of
    // the line passes per axis, pairs of real lines per CTA of the z passes
    int tile_line[3];
    int tile_z;
    // radix plan of the line passes per axis (0: built-in, 1: the alternative plan of the
    // type and length), chosen by the autotuner
    int line_variant[3];
    // FP32 and mixed: the three-pass schedule with fused plane passes (z and y transforms
    // of an x-plane in one cluster launch), where it exists; chosen by the autotuner
    bool plane_fused;
    // solves run as one persistent cooperative launch (sp_plan_set_persistent)
    bool persistent;
    // pass timing (diagnostic): events recorded between passes while timing is on.  The
    // events are a pool kept for the plan's life: ev_used of them hold the current record
    // ((npass + 1) per recorded solve); the pool grows only when a record outruns it.
    bool timing;
    int npass;                          // passes of one solve
    const char* pass_name[8];
    std::vector<cudaEvent_t>* ev;
    size_t ev_used;
    // Every member is a plain value or pointer, so a copy of the struct is a plain
    // byte copy that allocates nothing.
};

// Record a timing event on `st` if the plan is timing (no-op otherwise).
sp_status sp_mark(sp_plan p, cudaStream_t st);
// Record the plan's completion event on `st` after work issued there.
sp_status sp_record_done(sp_plan p, cudaStream_t st);
// Device allocation owned by the plan (the caller's allocator, else cudaMalloc).
// Host-built Bluestein table of one axis (layout above), in the plan's arithmetic type:
// bytes, and the fill into a host buffer of that size.
size_t sp_bluestein_bytes(const sp_plan_s* p, int ax);
void sp_bluestein_fill(const sp_plan_s* p, int ax, void* host);
sp_status sp_plan_alloc(sp_plan p, void** ptr, size_t bytes, const char* what);

// Thread-local error message helpers (sp_api.cu).
void sp_clear_error(void);
sp_status sp_fail(sp_status st, const char* fmt, ...);
sp_status sp_cuda_check(cudaError_t e, const char* what);
sp_status sp_check_device(const sp_plan p);  // SP_ERR_INVALID unless p's device is current

// Setup (sp_setup.cu).  All FP64.
sp_status sp_setup_run(sp_plan p, cudaStream_t st);
// Length of the generated GS table for the plan's eps and delta, and its exponents a_s
// (host, the same values the GPU generates up to rounding of exp).
int sp_gs_terms(const sp_plan p);
void sp_gs_exponents(const sp_plan p, double* a);

// Register-resident solve passes for the compiled lengths (sp_v2_*.cu); they return
// SP_ERR_UNSUPPORTED_SIZE, with no message, when an axis length has no compiled plan.
sp_status sp_v2_solve_f32(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st, bool mixed);
sp_status sp_v2_solve_f64(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st);
sp_status sp_v2_solve_df(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st);
sp_status sp_v2_forward_f32(sp_plan p, const void* rho, void* spec, cudaStream_t st, bool mixed);
sp_status sp_v2_forward_f64(sp_plan p, const void* rho, void* spec, cudaStream_t st);
sp_status sp_v2_forward_df(sp_plan p, const void* rho, void* spec, cudaStream_t st);
bool sp_v2_supported(int N);
// Double-float and FP32 plans keep, after the N base twiddles of an axis, the per-stage
// twiddle tables that their passes read from global memory; room for this many entries
// is reserved.
#define SP_TW_STAGED_MAX 8192
sp_status sp_v2_stage_twiddles_df(sp_plan p, cudaStream_t st);
sp_status sp_v2_stage_twiddles_f32(sp_plan p, cudaStream_t st);
sp_status sp_v2_persistent_f32(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st, bool mixed);
sp_status sp_v2_persistent_f64(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st);
sp_status sp_v2_persistent_df(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st);
float sp_v2_time_pass_f32(sp_plan p, int pass, int tile, int batch, int iters, cudaStream_t st, bool mixed, int variant);
float sp_v2_time_pass_f64(sp_plan p, int pass, int tile, int batch, int iters, cudaStream_t st, int variant);
float sp_v2_time_pass_df(sp_plan p, int pass, int tile, int batch, int iters, cudaStream_t st, int variant);
// radices of the register-resident passes in use: out[8 ax + s], ax = x, y, z passes
// whether the type has an alternative radix plan for the line passes at padded length N
bool sp_v2_has_alt_f32(int N);
bool sp_v2_plane_supported_f32(sp_plan p);
float sp_v2_time_solve_f32(sp_plan p, int batch, int iters, cudaStream_t st, bool mixed);
bool sp_v2_has_alt_df(int N);
sp_status sp_v2_radices_f32(sp_plan p, int* out);
sp_status sp_v2_radices_f64(sp_plan p, int* out);
sp_status sp_v2_radices_df(sp_plan p, int* out);

// Solve passes (sp_passes.cu).
sp_status sp_run_solve(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st);
sp_status sp_run_forward(sp_plan p, const void* rho, void* spec, cudaStream_t st);
