// Solve passes of Alg. 2 on the register-resident FFT engine (sp_fft.cuh), for padded
// lengths with a compile-time plan (64, 128, 192, 256, 384, 512, 1024).  The schedule
// and the workspace layout are those of the first-generation passes (sp_passes.cu):
//   z forward (packed real pairs) -> y forward -> x forward * M * x inverse
//   -> y inverse -> z inverse (packed real pairs), W[x][ky][kz] with row stride ldz.
// Included by one translation unit per arithmetic type (float, double, double-float).
#pragma once

#include <atomic>
#include <type_traits>

#include "sp_fft.cuh"
#include "sp_internal.h"

namespace v2 {

// ------------------------------------------------------------------ conversions
template <class R, class Tio> SP_D R to_r(Tio x);
template <> SP_D float to_r<float, float>(float x) { return x; }
template <> SP_D double to_r<double, double>(double x) { return x; }
template <> SP_D float to_r<float, double>(double x) { return (float)x; }
template <> SP_D df32 to_r<df32, double>(double x) { return df_from_double(x); }

template <class R, class Tio> SP_D Tio from_r(R x);
template <> SP_D float from_r<float, float>(float x) { return x; }
template <> SP_D double from_r<double, double>(double x) { return x; }
template <> SP_D double from_r<float, double>(float x) { return (double)x; }
template <> SP_D double from_r<df32, double>(df32 x) { return df_to_double(x); }

template <class R> SP_D cpx<R> half_of(cpx<R> a) { return scale(a, Num<R>::c(0.5)); }

// ------------------------------------------------------------------ layouts
// Strided lines: lane b (column) is fastest, B = 2^lgB columns per CTA (a runtime tile,
// handled with shifts and masks).  A padding row of B entries after every 8 rows keeps
// the stride-8 writes of the first stage off one bank set when a row of B entries is
// narrower than 128 bytes.
template <class R> struct LayStrided {
    int lgB, pad_mask, b;
    SP_D LayStrided(int lgB_, int b_)
        : lgB(lgB_), pad_mask(((1 << lgB_) * (int)sizeof(cpx<R>) >= 128) ? 0 : ~0), b(b_)
    {
    }
    SP_D int operator()(int e) const { return (e << lgB) + (((e >> 3) << lgB) & pad_mask) + b; }
    SP_D int unit() const { return 1 << lgB; }
    SP_D int step(int d) const { return (d << lgB) + (((d >> 3) << lgB) & pad_mask); }  // d a multiple of 8
    static constexpr SP_HD int size(int N, int B) { return N * B + (N / 8) * (B * (int)sizeof(cpx<R>) >= 128 ? 0 : B); }
};
// Contiguous lines: lane t is fastest; one padding entry after every 8 entries.
template <int N> struct LayLine {
    static constexpr int LD = N + N / 8;
    int base;
    SP_D int operator()(int e) const { return base + e + (e >> 3); }
    SP_D int unit() const { return 1; }
    SP_D int step(int d) const { return d + d / 8; }
};

// Shared memory of a pass: the staged twiddles of the directions it runs (unless they
// are read from global memory, below), then one or two exchange buffers (two when both
// fit in 100 KB, for one barrier per stage).  The twiddle entry count is rounded up to
// an even count, so that everything after it starts on a 16-byte boundary.
template <class R, int N> constexpr int tw_entries() { return (tw_stage_size<R, N>() + 1) & ~1; }
// Passes whose staged twiddles come from global memory (the plan's copy after its N base
// twiddles, cached in L1) rather than shared memory: double-float, whose tables (21 KB
// per CTA at 512, 56 KB at 1024) limit the resident CTAs and cost a fill per CTA
// (measured: 8 % faster at 128^3, 5 % at 256^3, 17 % at 512^3), and FP32 (its z passes
// 20-30 % faster).  The pipelined line kernel keeps its tables in shared memory.
template <class R, int N> constexpr bool tw_global() { return std::is_same<R, df32>::value || std::is_same<R, float>::value; }
template <class R, int N, class K = R> constexpr size_t pass_tw_bytes() { return tw_global<R, N>() ? 0 : sizeof(cpx<R>) * tw_entries<K, N>(); }

// Offset of plan key K's staged table after an axis's N base twiddles (entries).
template <class R, int N, class K> constexpr int tw_key_offset()
{
    if constexpr (KeyVariant<K>::v == 1) return tw_entries<R, N>();
    else return 0;
}
constexpr bool two_buffers(size_t buf_bytes, size_t tw_bytes) { return 2 * buf_bytes + tw_bytes <= 100 * 1024; }

// ------------------------------------------------------------------ strided passes
enum { FWD = 0, INV = 1, XMUL = 2 };

struct LArgs {
    const void* in;
    void* out;
    long long in_os, in_es, in_bs;  // outer / element / batch strides (complex elements)
    long long out_os, out_es, out_bs;
    int ncol;                        // valid columns (kz = 0..n2)
    int in_ld;                       // columns allocated per input row (>= ncol)
    int B;                           // columns per CTA (a power of two <= lanes_b_max<R, N>())
    int lgB;                         // log2(B), set by the launcher
    const void* tw;                  // exp(-2 pi i j / N), j < N
    const void* M;                   // XMUL: multiplier [|ko|][|kl|][kz], row stride ldzM
    int No, nh_line, ldzM;
    int reverse;                     // walk the outer index from the end: the previous pass
                                     // wrote its last outer indices last, so they are still in L2
};

// Largest column tile of a line pass (the launch bound of the runtime-tile kernel):
// 512 threads per CTA for 16-byte complex values (room for 128 registers), 1024 for
// 8-byte ones.
template <class R, int N> constexpr int lanes_b_max()
{
    return sizeof(cpx<R>) >= 16 ? (N >= 1024 ? 4 : 8) : (N >= 1024 ? 8 : 16);
}
template <int N> constexpr int lanes_b_default() { return N >= 1024 ? 4 : 8; }

// Resident CTAs per SM requested from the compiler: 1024 threads per SM (at most 64
// registers per thread) for the 8-value plans, to hide global-memory latency; the
// 24-value plans (lengths with a factor 3) keep their registers.
template <class K, int N, int THREADS> constexpr int min_blocks() { return PlanOf<K, N>::E <= 8 ? 1024 / THREADS : 1; }

// LGB >= 0: the tile 2^LGB is a compile-time constant (the default tile); LGB = -1: the
// tile comes from a.lgB (other tiles chosen by the autotuner).
template <class R, int N> constexpr int lg_max()
{
    return lanes_b_max<R, N>() >= 16 ? 4 : (lanes_b_max<R, N>() >= 8 ? 3 : 2);
}
template <class R, int N, int LGB, class K = R> constexpr int line_threads()
{
    return (N / PlanOf<K, N>::E) << (LGB >= 0 ? LGB : lg_max<R, N>());
}
template <int N> constexpr int lg_default() { return N >= 1024 ? 2 : 3; }

// ------------------------------------------------------------------ asynchronous copies
SP_D void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
SP_D void cp_async8(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
SP_D void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
SP_D void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// The x pass of the 8-byte-multiplier types (double-float, FP64) copies each thread's
// multiplier values into shared memory with cp.async when its tile starts, so the loads
// overlap the forward transform without holding registers; N B values of R per CTA.
template <class R, int MODE> constexpr bool stage_m() { return MODE == XMUL && sizeof(R) >= 8; }
template <class R, int N, int MODE> constexpr size_t stage_m_bytes(int B) { return stage_m<R, MODE>() ? sizeof(R) * (size_t)N * B : 0; }

// One tile of a line pass: B columns (c = cb B + b) of outer index o, right-hand side
// `batch`; all threads of the block take part.  `smraw` is the pass's dynamic shared
// memory (staged twiddles where they live in shared memory, then the exchange buffers).
template <class R, int N, int MODE, int LGB, class K = R>
SP_D void line_tile(const LArgs& a, int cb, int o, int batch, unsigned char* smraw)
{
    constexpr int E = PlanOf<K, N>::E, T = N / E;
    constexpr int R0 = PlanOf<K, N>::R[0];
    using Lay = LayStrided<R>;
    const int lgB = LGB >= 0 ? LGB : a.lgB, B = 1 << lgB;
    const int BUF = Lay::size(N, B);
    const bool DB = two_buffers(sizeof(cpx<R>) * BUF, pass_tw_bytes<R, N, K>());
    cpx<R>* tws_s = reinterpret_cast<cpx<R>*>(smraw);
    cpx<R>* sm0 = tws_s + pass_tw_bytes<R, N, K>() / sizeof(cpx<R>);
    cpx<R>* sm1 = DB ? sm0 + BUF : sm0;
    const int tid = threadIdx.x, b = tid & (B - 1), t = tid >> lgB;
    const cpx<R>* twg = static_cast<const cpx<R>*>(a.tw);
    const cpx<R>* tws = tw_global<R, N>() ? twg + N + tw_key_offset<R, N, K>() : tws_s;
    if constexpr (!tw_global<R, N>()) {
        if constexpr (MODE != INV) fill_stage_twiddles<R, N, false, K>(tws_s, twg, tid, blockDim.x);
        if constexpr (MODE != FWD) fill_stage_twiddles<R, N, true, K>(tws_s, twg, tid, blockDim.x);
    }
    const int c = cb * B + b;
    const bool cv = c < a.ncol;
    const cpx<R>* in = static_cast<const cpx<R>*>(a.in) + batch * a.in_bs + o * a.in_os + c;
    cpx<R>* out = static_cast<cpx<R>*>(a.out) + batch * a.out_bs + o * a.out_os + c;
    const Lay lay(lgB, b);
    cpx<R> v[E];
    if constexpr (MODE == INV) {
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int e = first_element<K, N, true>(t, j);
            v[j] = cv ? in[e * a.in_es] : czero<R>();
        }
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int e = first_element<K, N, false>(t, j);
            v[j] = (cv && (j % R0) < R0 / 2) ? in[e * a.in_es] : czero<R>();
        }
    }
    // x pass: the multiplier values of this thread's outputs are fetched before the forward
    // transform, so their latency overlaps its arithmetic: into registers for FP32, into
    // shared memory by cp.async for the 8-byte types (whose registers hold the transform)
    constexpr bool PREFETCH_M = MODE == XMUL && sizeof(R) == 4;
    constexpr bool STAGE_M = stage_m<R, MODE>();
    R mv[MODE == XMUL ? E : 1];
    const R* M = static_cast<const R*>(a.M);
    const int ko = o <= a.No / 2 ? o : a.No - o;
    const long long mrow = (long long)ko * (a.nh_line + 1);
    R* mst = reinterpret_cast<R*>(sm1 + BUF);  // STAGE_M: [j][thread]
    if constexpr (PREFETCH_M) {
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int e = last_element<K, N, false>(t, j);
            const int ke = e <= N / 2 ? e : N - e;
            mv[j] = cv ? M[(mrow + ke) * a.ldzM + c] : Num<R>::c(0.0);
        }
    } else if constexpr (STAGE_M) {
        if (cv) {
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const int e = last_element<K, N, false>(t, j);
                const int ke = e <= N / 2 ? e : N - e;
                cp_async8(&mst[j * blockDim.x + tid], &M[(mrow + ke) * a.ldzM + c]);
            }
        }
        cp_async_commit();
    }
    __syncthreads();
    cpx<R>* fresh;
    if constexpr (MODE == INV) {
        fresh = run_stages<R, N, true, +1, false, K>(v, sm0, sm1, lay, tws, t);
    } else {
        fresh = run_stages<R, N, false, -1, true, K>(v, sm0, sm1, lay, tws, t);
    }
    if constexpr (MODE == XMUL) {
        if constexpr (STAGE_M) cp_async_wait_all();  // this thread's own copies: no barrier needed
#pragma unroll
        for (int j = 0; j < E; ++j) {
            if constexpr (STAGE_M) {
                mv[j] = cv ? mst[j * blockDim.x + tid] : Num<R>::c(0.0);
            } else if constexpr (!PREFETCH_M) {
                const int e = last_element<K, N, false>(t, j);
                const int ke = e <= N / 2 ? e : N - e;
                mv[j] = cv ? M[(mrow + ke) * a.ldzM + c] : Num<R>::c(0.0);
            }
            v[j] = scale(v[j], mv[j]);
        }
        run_stages<R, N, true, +1, false, K>(v, fresh, fresh == sm0 ? sm1 : sm0, lay, tws, t);
    }
    if constexpr (MODE == FWD) {
#pragma unroll
        for (int j = 0; j < E; ++j)
            if (cv) out[last_element<K, N, false>(t, j) * a.out_es] = norm(v[j]);
    } else {  // the last inverse radix is R0: outputs q < R0/2 are the kept half
#pragma unroll
        for (int j = 0; j < E; ++j)
            if ((j % R0) < R0 / 2 && cv) out[last_element<K, N, true>(t, j) * a.out_es] = norm(v[j]);
    }
}

template <class R, int N, int MODE, int LGB, class K = R>
__global__ void __launch_bounds__(line_threads<R, N, LGB, K>(), LGB >= 0 ? min_blocks<K, N, line_threads<R, N, LGB, K>()>() : 1)
    k2_line(LArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    line_tile<R, N, MODE, LGB, K>(a, blockIdx.x, a.reverse ? gridDim.y - 1 - blockIdx.y : blockIdx.y, blockIdx.z, smraw);
}

// ------------------------------------------------------------------ pipelined line passes
// Persistent variant of k2_line (default tile only): each CTA walks tiles (batch, outer
// index, column block) with a stride of gridDim.x.  A tile's input rows (B contiguous
// complex values each) are copied into a shared-memory stage with cp.async; after the
// threads have moved the current tile's values from the stage into registers, the copies
// of the next tile are issued, so they land while the current tile computes.

struct PArgs {
    LArgs a;
    int outer;   // extent of the outer index
    int ncb;     // column blocks
    int ntiles;  // batch * outer * ncb
};

template <class R, int N, int MODE> constexpr int stage_rows() { return MODE == INV ? N : N / 2; }
// Two exchange buffers when they fit beside the twiddles and the stage in 110 KB (two CTAs
// per SM), else one.
// The y passes of the 32-value plan at 512 (one exchange a transform) trade the second
// buffer for a third resident CTA (measured: y passes 10 % faster; the 1024 passes are
// faster with two buffers and two CTAs).  So does the FP32 x pass of that plan, whose
// multiplier rows are then copied into shared memory by cp.async (one stage, refilled for
// the next tile right after the multiply) instead of being held in 32 registers a thread
// (measured: x pass 0.224 against 0.235 ms at 256^3; with two multiplier stages, which
// leave room for two CTAs only, or with the twiddles read from global memory instead of
// shared memory, it is slower than the register version).
template <class R, int N, int MODE, class K = R> constexpr bool pipe_mstage()
{
    return MODE == XMUL && std::is_same<R, float>::value && N <= 512 && PlanOf<K, N>::E >= 32;
}
template <class R, int N, int MODE, class K = R> constexpr bool pipe_third_cta()
{
    return (PlanOf<K, N>::E >= 32 && MODE != XMUL && N <= 512) || pipe_mstage<R, N, MODE, K>();
}
template <class R, int N, int MODE, class K = R> constexpr size_t pipe_mstage_bytes()
{
    return pipe_mstage<R, N, MODE, K>() ? sizeof(R) * (size_t)(N / 2 + 1) * (1 << lg_default<N>()) : 0;
}
template <class R, int N, int MODE, class K = R> constexpr bool pipe_two_buffers()
{
    constexpr int B = 1 << lg_default<N>();
    constexpr size_t buf = sizeof(cpx<R>) * (size_t)LayStrided<R>::size(N, B);
    constexpr size_t twb = sizeof(cpx<R>) * tw_entries<K, N>();
    return !pipe_third_cta<R, N, MODE, K>() &&
           twb + 2 * buf + sizeof(cpx<R>) * (size_t)stage_rows<R, N, MODE>() * B <= 110 * 1024;
}
template <class R, int N, int MODE, class K = R> constexpr size_t pipe_smem()
{
    constexpr int B = 1 << lg_default<N>();
    constexpr size_t buf = sizeof(cpx<R>) * (size_t)LayStrided<R>::size(N, B);
    constexpr size_t twb = sizeof(cpx<R>) * tw_entries<K, N>();
    return twb + (pipe_two_buffers<R, N, MODE, K>() ? 2 : 1) * buf + sizeof(cpx<R>) * (size_t)stage_rows<R, N, MODE>() * B +
           pipe_mstage_bytes<R, N, MODE, K>();
}

template <class R, int N, int MODE, class K = R>
__global__ void __launch_bounds__(line_threads<R, N, lg_default<N>(), K>(),
                                  pipe_third_cta<R, N, MODE, K>() ? 3 : min_blocks<K, N, line_threads<R, N, lg_default<N>(), K>()>())
    k3_line(PArgs pa)
{
    constexpr int E = PlanOf<K, N>::E, T = N / E;
    constexpr int R0 = PlanOf<K, N>::R[0];
    constexpr int LGB = lg_default<N>(), B = 1 << LGB;
    constexpr int NIN = stage_rows<R, N, MODE>();
    constexpr int CH = B * (int)sizeof(cpx<R>) / 16;  // 16-byte chunks per row
    using Lay = LayStrided<R>;
    constexpr bool MST = pipe_mstage<R, N, MODE, K>();
    constexpr int MROWS = N / 2 + 1;              // MST: multiplier rows |kx| = 0 .. N/2
    constexpr int MCH = B * (int)sizeof(R) / 16;  // MST: 16-byte chunks per multiplier row
    // cp.async writes 16-byte chunks: the stage must start on a 16-byte boundary
    static_assert((sizeof(cpx<R>) * tw_entries<K, N>()) % 16 == 0, "twiddle area alignment");
    static_assert((sizeof(cpx<R>) * Lay::size(N, B)) % 16 == 0, "exchange buffer alignment");
    static_assert((B * sizeof(cpx<R>)) % 16 == 0, "stage row alignment");
    static_assert(!MST || (B * sizeof(R)) % 16 == 0, "multiplier stage alignment");
    const LArgs& a = pa.a;
    const int BUF = Lay::size(N, B);
    constexpr bool DB = pipe_two_buffers<R, N, MODE, K>();
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<R>* tws = reinterpret_cast<cpx<R>*>(smraw);
    cpx<R>* sm0 = tws + tw_entries<K, N>();
    cpx<R>* sm1 = DB ? sm0 + BUF : sm0;
    cpx<R>* stg = sm0 + (DB ? 2 : 1) * BUF;
    R* mstg = reinterpret_cast<R*>(stg + NIN * B);  // MST: [|kx|][column of the tile]
    const int tid = threadIdx.x, b = tid & (B - 1), t = tid >> LGB;
    const cpx<R>* twg = static_cast<const cpx<R>*>(a.tw);
    if constexpr (MODE != INV) fill_stage_twiddles<R, N, false, K>(tws, twg, tid, blockDim.x);
    if constexpr (MODE != FWD) fill_stage_twiddles<R, N, true, K>(tws, twg, tid, blockDim.x);
    const Lay lay(LGB, b);
    // tile index = (batch * outer + o) * ncb + cb.  The first tile is decoded by division;
    // each later one adds gridDim.x in that mixed radix (two compares, no division).
    struct TileIdx {
        int batch, o, cb;
    };
    const int g_cb = (int)gridDim.x % pa.ncb, g_r = (int)gridDim.x / pa.ncb;
    const int g_o = g_r % pa.outer, g_b = g_r / pa.outer;
    auto advance = [&](TileIdx x) {
        x.cb += g_cb;
        int carry = x.cb >= pa.ncb;
        if (carry) x.cb -= pa.ncb;
        x.o += g_o + carry;
        carry = x.o >= pa.outer;
        if (carry) x.o -= pa.outer;
        x.batch += g_b + carry;
        return x;
    };
    auto issue = [&](TileIdx x) {
        const int xo = a.reverse ? pa.outer - 1 - x.o : x.o;
        const char* src = reinterpret_cast<const char*>(static_cast<const cpx<R>*>(a.in) + x.batch * a.in_bs +
                                                        xo * a.in_os + x.cb * B);
        for (int q = tid; q < NIN * CH; q += blockDim.x) {
            const int row = q / CH, ch = q % CH;
            cp_async16(reinterpret_cast<char*>(stg) + (size_t)row * B * sizeof(cpx<R>) + ch * 16,
                       src + (long long)row * a.in_es * (long long)sizeof(cpx<R>) + ch * 16);
        }
        cp_async_commit();
    };
    // MST: the tile's multiplier rows M[|ky|][|kx|][c0 .. c0 + B), |kx| = 0 .. N/2
    auto issue_m = [&](TileIdx x) {
        const int xo = a.reverse ? pa.outer - 1 - x.o : x.o;
        const int ko = xo <= a.No / 2 ? xo : a.No - xo;
        const char* src = reinterpret_cast<const char*>(static_cast<const R*>(a.M) +
                                                        (long long)ko * (a.nh_line + 1) * a.ldzM + x.cb * B);
        for (int q = tid; q < MROWS * MCH; q += blockDim.x) {
            const int row = q / MCH, ch = q % MCH;
            cp_async16(reinterpret_cast<char*>(mstg) + (size_t)row * B * sizeof(R) + ch * 16,
                       src + (long long)row * a.ldzM * (long long)sizeof(R) + ch * 16);
        }
    };
    TileIdx cur;
    cur.cb = (int)blockIdx.x % pa.ncb;
    cur.o = ((int)blockIdx.x / pa.ncb) % pa.outer;
    cur.batch = ((int)blockIdx.x / pa.ncb) / pa.outer;
    if (blockIdx.x < pa.ntiles) {
        if constexpr (MST) issue_m(cur);  // committed with the rows
        issue(cur);
    }
    for (int tile = blockIdx.x; tile < pa.ntiles; tile += gridDim.x) {
        const TileIdx nxt = advance(cur);
        const int batch = cur.batch, o = a.reverse ? pa.outer - 1 - cur.o : cur.o, cb = cur.cb;
        const int c = cb * B + b;
        const bool cv = c < a.ncol;
        cp_async_wait_all();
        __syncthreads();  // this tile's rows (and, on the first tile, the twiddles) are in
        cpx<R> v[E];
        if constexpr (MODE == INV) {
#pragma unroll
            for (int j = 0; j < E; ++j) v[j] = stg[first_element<K, N, true>(t, j) * B + b];
        } else {
#pragma unroll
            for (int j = 0; j < E; ++j)
                v[j] = ((j % R0) < R0 / 2) ? stg[first_element<K, N, false>(t, j) * B + b] : czero<R>();
        }
        constexpr bool PREFETCH_M = MODE == XMUL && sizeof(R) == 4 && !MST;
        R mv[MODE == XMUL ? E : 1];
        const R* M = static_cast<const R*>(a.M);
        const int ko = o <= a.No / 2 ? o : a.No - o;
        const long long mrow = (long long)ko * (a.nh_line + 1);
        if constexpr (PREFETCH_M) {
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const int e = last_element<K, N, false>(t, j);
                const int ke = e <= N / 2 ? e : N - e;
                mv[j] = cv ? M[(mrow + ke) * a.ldzM + c] : Num<R>::c(0.0);
            }
        }
        __syncthreads();  // the stage is free: start the next tile's copies
        if (tile + (int)gridDim.x < pa.ntiles) issue(nxt);
        cpx<R>* fresh;
        if constexpr (MODE == INV) {
            fresh = run_stages<R, N, true, +1, false, K>(v, sm0, sm1, lay, tws, t);
        } else {
            fresh = run_stages<R, N, false, -1, true, K>(v, sm0, sm1, lay, tws, t);
        }
        if constexpr (MODE == XMUL) {
#pragma unroll
            for (int j = 0; j < E; ++j) {
                if constexpr (MST) {
                    const int e = last_element<K, N, false>(t, j);
                    const int ke = e <= N / 2 ? e : N - e;
                    mv[j] = cv ? mstg[ke * B + b] : Num<R>::c(0.0);
                } else if constexpr (!PREFETCH_M) {
                    const int e = last_element<K, N, false>(t, j);
                    const int ke = e <= N / 2 ? e : N - e;
                    mv[j] = cv ? M[(mrow + ke) * a.ldzM + c] : Num<R>::c(0.0);
                }
                v[j] = scale(v[j], mv[j]);
            }
            if constexpr (MST) {  // every thread has read the stage: refill it for the next tile
                if (tile + (int)gridDim.x < pa.ntiles) {
                    __syncthreads();
                    issue_m(nxt);
                    cp_async_commit();
                }
            }
            run_stages<R, N, true, +1, false, K>(v, fresh, fresh == sm0 ? sm1 : sm0, lay, tws, t);
        }
        cpx<R>* out = static_cast<cpx<R>*>(a.out) + batch * a.out_bs + o * a.out_os + c;
        if constexpr (MODE == FWD) {
#pragma unroll
            for (int j = 0; j < E; ++j)
                if (cv) out[last_element<K, N, false>(t, j) * a.out_es] = norm(v[j]);
        } else {
#pragma unroll
            for (int j = 0; j < E; ++j)
                if ((j % R0) < R0 / 2 && cv) out[last_element<K, N, true>(t, j) * a.out_es] = norm(v[j]);
        }
        __syncthreads();  // exchange buffers free before the next tile's first write
        cur = nxt;
    }
    cp_async_wait_all();
}

// ------------------------------------------------------------------ z passes
struct ZArgs2 {
    const void* rho;
    void* u;
    void* W;
    int n1, n2;
    long long lines;      // n0 n1 real lines
    long long plane;      // complex elements per x-plane of W
    int ldz;
    long long io_bs, w_bs;
    const void* tw;
    int B;                // pairs of real lines per CTA (pairs_max<N>() / 2^j)
    int reverse;          // walk the lines from the end (their planes were written last by the
                          // previous pass, so they are still in L2)
};

template <int N> constexpr int pairs_max() { return N >= 512 ? 8 : (N >= 256 ? 16 : 32); }
template <int N> constexpr int pairs_default() { return N >= 512 ? 4 : (N >= 256 ? 8 : 16); }

SP_D long long w_row(const ZArgs2& a, long long l) { return (l / a.n1) * a.plane + (l % a.n1) * a.ldz; }

template <class R, int N> SP_HD int z_buf(int B) { return B * LayLine<N>::LD; }
template <class R, int N> SP_HD bool z_two_buffers(int B)
{
    return two_buffers(sizeof(cpx<R>) * z_buf<R, N>(B), pass_tw_bytes<R, N, ZKey<R>>());
}

// One tile of the z forward pass: a.B pairs of real lines starting at pair block `blk`,
// right-hand side `batch`.
template <class R, class Tio, int N>
SP_D void zf_tile(const ZArgs2& a, int blk, int batch, unsigned char* smraw)
{
    constexpr int E = PlanOf<ZKey<R>, N>::E, T = N / E;
    const int B = a.B;
    constexpr int R0 = PlanOf<ZKey<R>, N>::R[0];
    cpx<R>* tws_s = reinterpret_cast<cpx<R>*>(smraw);
    cpx<R>* sm0 = tws_s + pass_tw_bytes<R, N, ZKey<R>>() / sizeof(cpx<R>);
    cpx<R>* sm1 = z_two_buffers<R, N>(B) ? sm0 + z_buf<R, N>(B) : sm0;
    const int tid = threadIdx.x, b = tid / T, t = tid % T;
    const cpx<R>* tws = tw_global<R, N>() ? static_cast<const cpx<R>*>(a.tw) + N : tws_s;
    if constexpr (!tw_global<R, N>()) fill_stage_twiddles<R, N, false, ZKey<R>>(tws_s, static_cast<const cpx<R>*>(a.tw), tid, blockDim.x);
    const int n2 = a.n2;
    const long long l0 = 2 * ((long long)blk * B + b), l1 = l0 + 1;
    const Tio* rho = static_cast<const Tio*>(a.rho) + batch * a.io_bs;
    cpx<R>* W = static_cast<cpx<R>*>(a.W) + batch * a.w_bs;
    const LayLine<N> lay{b * LayLine<N>::LD};
    cpx<R> v[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int z = first_element<ZKey<R>, N, false>(t, j);
        R xr = Num<R>::c(0.0), xi = Num<R>::c(0.0);
        if ((j % R0) < R0 / 2) {  // z < n2: the padded half is zero
            if (l0 < a.lines) xr = to_r<R, Tio>(rho[l0 * n2 + z]);
            if (l1 < a.lines) xi = to_r<R, Tio>(rho[l1 * n2 + z]);
        }
        v[j] = mk(xr, xi);
    }
    __syncthreads();
    cpx<R>* sm = run_stages<R, N, false, -1, true, ZKey<R>>(v, sm0, sm1, lay, tws, t);
#pragma unroll
    for (int j = 0; j < E; ++j) sm[lay(last_element<ZKey<R>, N, false>(t, j))] = v[j];
    __syncthreads();
    // two real lines from one complex transform: Xa = (Z_k + conj Z_{N-k}) / 2,
    // Xb = (Z_k - conj Z_{N-k}) / (2 i), k = 0..n2
    const long long r0 = w_row(a, l0), r1 = w_row(a, l1 < a.lines ? l1 : l0);
    for (int k = t; k <= n2; k += T) {
        const cpx<R> zk = sm[lay(k)];
        const cpx<R> zm = conjg(sm[lay(k == 0 ? 0 : N - k)]);
        const cpx<R> s = zk + zm, d = zk - zm;
        if (l0 < a.lines) W[r0 + k] = norm(half_of(s));
        if (l1 < a.lines) W[r1 + k] = norm(half_of(mk(im_of(d), -re_of(d))));
    }
}

template <class R, class Tio, int N>
__global__ void __launch_bounds__((N / PlanOf<ZKey<R>, N>::E) * pairs_max<N>(),
                                  min_blocks<ZKey<R>, N, (N / PlanOf<ZKey<R>, N>::E) * pairs_max<N>()>()) k2_z_fwd(ZArgs2 a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    zf_tile<R, Tio, N>(a, a.reverse ? gridDim.x - 1 - blockIdx.x : blockIdx.x, blockIdx.y, smraw);
}

// One tile of the z inverse pass (pairs of real output lines), as zf_tile.
template <class R, class Tio, int N>
SP_D void zi_tile(const ZArgs2& a, int blk, int batch, unsigned char* smraw)
{
    constexpr int E = PlanOf<ZKey<R>, N>::E, T = N / E;
    const int B = a.B;
    constexpr int R0 = PlanOf<ZKey<R>, N>::R[0];
    cpx<R>* tws_s = reinterpret_cast<cpx<R>*>(smraw);
    cpx<R>* sm0 = tws_s + pass_tw_bytes<R, N, ZKey<R>>() / sizeof(cpx<R>);
    cpx<R>* sm1 = z_two_buffers<R, N>(B) ? sm0 + z_buf<R, N>(B) : sm0;
    const int tid = threadIdx.x, b = tid / T, t = tid % T;
    const cpx<R>* tws = tw_global<R, N>() ? static_cast<const cpx<R>*>(a.tw) + N : tws_s;
    if constexpr (!tw_global<R, N>()) fill_stage_twiddles<R, N, true, ZKey<R>>(tws_s, static_cast<const cpx<R>*>(a.tw), tid, blockDim.x);
    const int n2 = a.n2;
    const long long l0 = 2 * ((long long)blk * B + b), l1 = l0 + 1;
    Tio* u = static_cast<Tio*>(a.u) + batch * a.io_bs;
    const cpx<R>* W = static_cast<const cpx<R>*>(a.W) + batch * a.w_bs;
    const LayLine<N> lay{b * LayLine<N>::LD};
    // Z_k = Xa_k + i Xb_k from the Hermitian halves (DC and Nyquist take real parts)
    const long long r0 = w_row(a, l0), r1 = w_row(a, l1 < a.lines ? l1 : l0);
    for (int k = t; k <= n2; k += T) {
        const cpx<R> xa = l0 < a.lines ? W[r0 + k] : czero<R>();
        const cpx<R> xb = l1 < a.lines ? W[r1 + k] : czero<R>();
        const R ar = re_of(xa), br = re_of(xb);
        const bool edge = k == 0 || k == n2;
        const R ai = edge ? Num<R>::c(0.0) : im_of(xa), bi = edge ? Num<R>::c(0.0) : im_of(xb);
        sm0[lay(k)] = mk(ar - bi, ai + br);
        if (k > 0 && k < n2) sm0[lay(N - k)] = mk(ar + bi, br - ai);
    }
    __syncthreads();
    cpx<R> v[E];
    Stage<R, N, true, 0, ZKey<R>>::load(v, sm0, lay, t);
    if (sm1 == sm0) __syncthreads();
    run_stages<R, N, true, +1, false, ZKey<R>>(v, sm1, sm0, lay, tws, t);
#pragma unroll
    for (int j = 0; j < E; ++j) {
        if ((j % R0) < R0 / 2) {  // z < n2
            const int z = last_element<ZKey<R>, N, true>(t, j);
            if (l0 < a.lines) u[l0 * n2 + z] = from_r<R, Tio>(re_of(v[j]));
            if (l1 < a.lines) u[l1 * n2 + z] = from_r<R, Tio>(im_of(v[j]));
        }
    }
}

template <class R, class Tio, int N>
__global__ void __launch_bounds__((N / PlanOf<ZKey<R>, N>::E) * pairs_max<N>(),
                                  min_blocks<ZKey<R>, N, (N / PlanOf<ZKey<R>, N>::E) * pairs_max<N>()>()) k2_z_inv(ZArgs2 a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    zi_tile<R, Tio, N>(a, a.reverse ? gridDim.x - 1 - blockIdx.x : blockIdx.x, blockIdx.y, smraw);
}

// ------------------------------------------------------------------ launchers
// Raise one kernel's dynamic shared-memory limit once per device (the attribute is a
// per-device setting), to more than any of its launches uses, so that later launches
// (e.g. under stream capture) make no attribute call.
template <auto KERNEL> inline sp_status smem_attr(size_t bytes)
{
    static std::atomic<unsigned long long> done{0};  // bit d: set on device d
    if (bytes <= 48 * 1024) return SP_OK;
    int dev = 0;
    sp_status rc = sp_cuda_check(cudaGetDevice(&dev), "current device");
    if (rc) return rc;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_relaxed) & bit)) return SP_OK;
    rc = sp_cuda_check(cudaFuncSetAttribute(KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024),
                       "set shared memory size");
    if (rc == SP_OK) done.fetch_or(bit, std::memory_order_relaxed);
    return rc;
}

template <class R, int N, int MODE, class K = R>
sp_status launch_line(const LArgs& a, int outer, int batch, cudaStream_t st)
{
    constexpr int E = PlanOf<K, N>::E;
    LArgs ab = a;
    ab.B = a.B ? a.B : lanes_b_default<N>();
    const int B = ab.B;
    if (B < 1 || B > lanes_b_max<R, N>() || (B & (B - 1))) return sp_fail(SP_ERR_INVALID, "bad line tile %d", B);
    ab.lgB = 0;
    while ((1 << ab.lgB) < B) ++ab.lgB;
    const size_t buf = sizeof(cpx<R>) * LayStrided<R>::size(N, B);
    const size_t twb = pass_tw_bytes<R, N, K>();
    const size_t smem = twb + (two_buffers(buf, twb) ? 2 : 1) * buf + stage_m_bytes<R, N, MODE>(B);
    dim3 grid((unsigned)((a.ncol + B - 1) / B), (unsigned)outer, (unsigned)batch);
    sp_status rc;
    constexpr size_t psmem = pipe_smem<R, N, MODE, K>();
    // pipelined persistent kernel: default tile, inputs whose rows are 16-byte aligned
    // (the workspace), and a stage that still leaves two CTAs per SM
    const bool rows_aligned = ((uintptr_t)a.in % 16 == 0) && (a.in_es * sizeof(cpx<R>)) % 16 == 0 &&
                              (a.in_os * sizeof(cpx<R>)) % 16 == 0 && (a.in_bs * sizeof(cpx<R>)) % 16 == 0;
    // the staged multiplier rows are copied in 16-byte chunks as well
    const bool m_aligned = !pipe_mstage<R, N, MODE, K>() ||
                           ((uintptr_t)a.M % 16 == 0 && (a.ldzM * sizeof(R)) % 16 == 0 && (a.ncol + B - 1) / B * B <= a.ldzM);
    if (ab.lgB == lg_default<N>() && psmem <= 110 * 1024 && rows_aligned && m_aligned &&
        (a.ncol + B - 1) / B * B <= a.in_ld) {
        if ((rc = smem_attr<k3_line<R, N, MODE, K>>(psmem))) return rc;
        static std::atomic<int> per_sm_cached{0};  // resident CTAs per SM (same on every GB300)
        int per_sm = per_sm_cached.load(std::memory_order_relaxed);
        if (!per_sm) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k3_line<R, N, MODE, K>, (N / E) * B, psmem);
            if (per_sm < 1) per_sm = 1;
            per_sm_cached.store(per_sm, std::memory_order_relaxed);
        }
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        PArgs pa;
        pa.a = ab;
        pa.outer = outer;
        pa.ncb = (a.ncol + B - 1) / B;
        pa.ntiles = batch * outer * pa.ncb;
        const int nblocks = pa.ntiles < per_sm * sms ? pa.ntiles : per_sm * sms;
        k3_line<R, N, MODE, K><<<nblocks, (N / E) * B, psmem, st>>>(pa);
    } else if (ab.lgB == lg_default<N>()) {
        if ((rc = smem_attr<k2_line<R, N, MODE, lg_default<N>(), K>>(smem))) return rc;
        k2_line<R, N, MODE, lg_default<N>(), K><<<grid, (N / E) * B, smem, st>>>(ab);
    } else {
        if ((rc = smem_attr<k2_line<R, N, MODE, -1, K>>(smem))) return rc;
        k2_line<R, N, MODE, -1, K><<<grid, (N / E) * B, smem, st>>>(ab);
    }
    return sp_cuda_check(cudaGetLastError(), "v2 line pass");
}

template <class R, class Tio, int N>
sp_status launch_z(const ZArgs2& a, bool forward, int batch, cudaStream_t st)
{
    constexpr int E = PlanOf<ZKey<R>, N>::E;
    ZArgs2 ab = a;
    ab.B = a.B ? a.B : pairs_default<N>();
    const int B = ab.B;
    if (B < 1 || B > pairs_max<N>() || (pairs_max<N>() % B)) return sp_fail(SP_ERR_INVALID, "bad z tile %d", B);
    const size_t smem = pass_tw_bytes<R, N, ZKey<R>>() + sizeof(cpx<R>) * (z_two_buffers<R, N>(B) ? 2 : 1) * z_buf<R, N>(B);
    const long long pairs = (a.lines + 1) / 2;
    dim3 grid((unsigned)((pairs + B - 1) / B), (unsigned)batch);
    sp_status rc;
    if (forward) {
        if ((rc = smem_attr<k2_z_fwd<R, Tio, N>>(smem))) return rc;
        k2_z_fwd<R, Tio, N><<<grid, (N / E) * B, smem, st>>>(ab);
    } else {
        if ((rc = smem_attr<k2_z_inv<R, Tio, N>>(smem))) return rc;
        k2_z_inv<R, Tio, N><<<grid, (N / E) * B, smem, st>>>(ab);
    }
    return sp_cuda_check(cudaGetLastError(), forward ? "v2 z forward pass" : "v2 z inverse pass");
}

// Length dispatch: calls f.template run<N>() for a supported N.
template <class R, int N, class K>
__global__ void k_stage_twiddles(cpx<R>* dst, const cpx<R>* __restrict__ tw)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    fill_stage_twiddles<R, N, false, K>(dst, tw, tid, nth);
    fill_stage_twiddles<R, N, true, K>(dst, tw, tid, nth);
}

template <class F> inline sp_status with_len(int N, F&& f);

// K: the plan key of the passes that read the table (R and, where it exists, the
// alternative LineKey<R, 1> for the line passes; ZKey<R> for the z passes).
template <class R, class K> struct StageTw {
    cpx<R>* tw;
    cudaStream_t st;
    template <int N> sp_status run()
    {
        if constexpr (tw_global<R, N>() && (KeyVariant<K>::v == 0 || AltPlan<R, N>::exists)) {
            static_assert(tw_key_offset<R, N, K>() + tw_stage_size<K, N>() <= SP_TW_STAGED_MAX, "staged twiddle room");
            k_stage_twiddles<R, N, K><<<16, 256, 0, st>>>(tw + N + tw_key_offset<R, N, K>(), tw);
            return sp_cuda_check(cudaGetLastError(), "staged twiddles");
        }
        return SP_OK;
    }
};

template <class F> inline sp_status with_len(int N, F&& f)
{
    switch (N) {
        case 64: return f.template run<64>();
        case 128: return f.template run<128>();
        case 192: return f.template run<192>();
        case 256: return f.template run<256>();
        case 384: return f.template run<384>();
        case 512: return f.template run<512>();
        case 1024: return f.template run<1024>();
        default: return SP_ERR_UNSUPPORTED_SIZE;
    }
}

inline bool len_ok(int N)
{
    return N == 64 || N == 128 || N == 192 || N == 256 || N == 384 || N == 512 || N == 1024;
}

// variant 1: the alternative radix plan of this type and length (AltPlan), where it exists
template <class R, int MODE> struct LineRun {
    const LArgs* a;
    int outer, batch;
    cudaStream_t st;
    int variant;
    template <int N> sp_status run()
    {
        if constexpr (AltPlan<R, N>::exists) {
            if (variant) return launch_line<R, N, MODE, LineKey<R, 1>>(*a, outer, batch, st);
        } else {
            if (variant) return sp_fail(SP_ERR_UNSUPPORTED_SIZE, "no alternative radix plan for length %d", N);
        }
        return launch_line<R, N, MODE>(*a, outer, batch, st);
    }
};

// Radices of the plans a solve uses: out[8 ax + s] for stage s of axis ax's passes (the
// x pass, the y passes, the z passes), 0 after the last stage.
template <class K, int N> void copy_radices(int* out)
{
    for (int s = 0; s < 8; ++s) out[s] = s < PlanOf<K, N>::NS ? PlanOf<K, N>::R[s] : 0;
}
template <class R> struct RadicesOf {
    int* out;
    int variant;  // -1: the z passes' plan
    template <int N> sp_status run()
    {
        if (variant < 0) {
            copy_radices<ZKey<R>, N>(out);
        } else {
            if constexpr (AltPlan<R, N>::exists) {
                if (variant) {
                    copy_radices<LineKey<R, 1>, N>(out);
                    return SP_OK;
                }
            }
            copy_radices<R, N>(out);
        }
        return SP_OK;
    }
};
template <class R> sp_status radices(sp_plan p, int* out)
{
    sp_status rc;
    for (int ax = 0; ax < 2; ++ax)
        if ((rc = with_len(p->N[ax], RadicesOf<R>{out + 8 * ax, p->line_variant[ax]}))) return rc;
    return with_len(p->N[2], RadicesOf<R>{out + 16, -1});
}

template <class R, class Tio> struct ZRun {
    const ZArgs2* a;
    bool forward;
    int batch;
    cudaStream_t st;
    template <int N> sp_status run() { return launch_z<R, Tio, N>(*a, forward, batch, st); }
};

// Tables of the pass arithmetic type.
template <class R> struct Tabs {
    static const void* tw(sp_plan p, int ax);
    static const void* M(sp_plan p);
};

// Staged twiddle tables in global memory for the axes whose line passes read them there.
template <class R> sp_status stage_twiddles(sp_plan p, cudaStream_t st)
{
    for (int ax = 0; ax < 3; ++ax) {
        if (!len_ok(p->N[ax])) continue;
        cpx<R>* tw = static_cast<cpx<R>*>(const_cast<void*>(Tabs<R>::tw(p, ax)));
        sp_status rc = ax == 2 ? with_len(p->N[ax], StageTw<R, ZKey<R>>{tw, st}) : with_len(p->N[ax], StageTw<R, R>{tw, st});
        if (rc) return rc;
        if (ax < 2 && (rc = with_len(p->N[ax], StageTw<R, LineKey<R, 1>>{tw, st}))) return rc;
    }
    return SP_OK;
}

// The whole solve; `work` is the workspace (the plan's, or another of the same size).
template <class R, class Tio>
sp_status solve(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st, bool mark)
{
    for (int ax = 0; ax < 3; ++ax)
        if (!len_ok(p->N[ax])) return SP_ERR_UNSUPPORTED_SIZE;
    sp_status rc;
    p->npass = 5;
    p->pass_name[0] = "z_forward";
    p->pass_name[1] = "y_forward";
    p->pass_name[2] = "x_multiply";
    p->pass_name[3] = "y_inverse";
    p->pass_name[4] = "z_inverse";
    ZArgs2 z = {};
    z.rho = rho;
    z.u = u;
    z.W = p->d_work;
    z.n1 = p->n[1];
    z.n2 = p->n[2];
    z.lines = (long long)p->n[0] * p->n[1];
    z.plane = p->plane;
    z.ldz = p->ldz;
    z.io_bs = (long long)p->n[0] * p->n[1] * p->n[2];
    z.w_bs = (long long)p->n[0] * p->plane;
    z.tw = Tabs<R>::tw(p, 2);
    z.B = p->tile_z;
    LArgs y = {};
    y.in = y.out = p->d_work;
    y.in_os = y.out_os = p->plane;
    y.in_es = y.out_es = p->ldz;
    y.in_bs = y.out_bs = (long long)p->n[0] * p->plane;
    y.ncol = p->n[2] + 1;
    y.in_ld = p->ldz;
    y.tw = Tabs<R>::tw(p, 1);
    y.B = p->tile_line[1];
    LArgs x = y;
    x.in_os = x.out_os = p->ldz;
    x.in_es = x.out_es = p->plane;
    x.tw = Tabs<R>::tw(p, 0);
    x.M = Tabs<R>::M(p);
    x.B = p->tile_line[0];
    x.No = p->N[1];
    x.nh_line = p->n[0];
    x.ldzM = p->ldz;
    // Each pass writes its outer indices in increasing order, so what it wrote last is still
    // in L2 when the next pass starts: the y forward pass walks the planes the z forward
    // pass wrote from the last one down, and the z inverse pass the rows the y inverse pass
    // wrote (the x pass reads every plane in every tile, so its order does not matter).
    LArgs yf = y, yi = y;
    yf.reverse = 1;
    ZArgs2 zf = z, zi = z;
    zi.reverse = 1;
    if (mark && (rc = sp_mark(p, st))) return rc;
    if ((rc = with_len(p->N[2], ZRun<R, Tio>{&zf, true, batch, st}))) return rc;
    if (mark && (rc = sp_mark(p, st))) return rc;
    if ((rc = with_len(p->N[1], LineRun<R, FWD>{&yf, p->n[0], batch, st, p->line_variant[1]}))) return rc;
    if (mark && (rc = sp_mark(p, st))) return rc;
    if ((rc = with_len(p->N[0], LineRun<R, XMUL>{&x, p->N[1], batch, st, p->line_variant[0]}))) return rc;
    if (mark && (rc = sp_mark(p, st))) return rc;
    if ((rc = with_len(p->N[1], LineRun<R, INV>{&yi, p->n[0], batch, st, p->line_variant[1]}))) return rc;
    if (mark && (rc = sp_mark(p, st))) return rc;
    if ((rc = with_len(p->N[2], ZRun<R, Tio>{&zi, false, batch, st}))) return rc;
    if (mark && (rc = sp_mark(p, st))) return rc;
    return SP_OK;
}

// Time `iters` launches of one pass (0: z passes, 1: y passes, 2: x pass) with the
// given tile, on the plan's workspace (contents irrelevant: the arithmetic does not
// depend on the data), `batch` right-hand sides (the z passes of every right-hand side
// read and write one dummy input and output inside the workspace, the line passes their
// own workspace slices, as in the solve).  Host-synchronising.  Returns the mean
// milliseconds per launch, or a negative value on error.
template <class R, class Tio>
float time_pass(sp_plan p, int pass, int tile, int batch, int iters, cudaStream_t st, int variant)
{
    ZArgs2 z = {};
    z.rho = p->d_work;
    z.u = (char*)p->d_work + p->work_bytes / 2;  // the z passes only need valid addresses
    z.W = p->d_work;
    z.n1 = p->n[1];
    z.n2 = p->n[2];
    z.lines = (long long)p->n[0] * p->n[1];
    z.plane = p->plane;
    z.ldz = p->ldz;
    z.io_bs = 0;
    z.w_bs = (long long)p->n[0] * p->plane;
    z.tw = Tabs<R>::tw(p, 2);
    z.B = tile;
    LArgs y = {};
    y.in = y.out = p->d_work;
    y.in_os = y.out_os = p->plane;
    y.in_es = y.out_es = p->ldz;
    y.in_bs = y.out_bs = (long long)p->n[0] * p->plane;
    y.ncol = p->n[2] + 1;
    y.in_ld = p->ldz;
    y.tw = Tabs<R>::tw(p, 1);
    y.B = tile;
    LArgs x = y;
    x.in_os = x.out_os = p->ldz;
    x.in_es = x.out_es = p->plane;
    x.tw = Tabs<R>::tw(p, 0);
    x.M = Tabs<R>::M(p);
    x.No = p->N[1];
    x.nh_line = p->n[0];
    x.ldzM = p->ldz;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return -1.f; }
    sp_status rc = SP_OK;
    for (int it = -1; it < iters && rc == SP_OK; ++it) {  // it = -1: warm-up launch
        if (it == 0) cudaEventRecord(e0, st);
        if (pass == 0) {  // every right-hand side reads the same input and writes the same output
            rc = with_len(p->N[2], ZRun<R, Tio>{&z, true, batch, st});
            if (rc == SP_OK) rc = with_len(p->N[2], ZRun<R, Tio>{&z, false, batch, st});
        } else if (pass == 1) {
            rc = with_len(p->N[1], LineRun<R, FWD>{&y, p->n[0], batch, st, variant});
            if (rc == SP_OK) rc = with_len(p->N[1], LineRun<R, INV>{&y, p->n[0], batch, st, variant});
        } else {
            rc = with_len(p->N[0], LineRun<R, XMUL>{&x, p->N[1], batch, st, variant});
        }
    }
    cudaEventRecord(e1, st);
    float ms = -1.f;
    if (rc == SP_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
        ms /= iters;
    else
        ms = -1.f;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

// ------------------------------------------------------------------ persistent solve
// All five passes of a (batched) solve in one cooperative launch: every block walks the
// tiles of a pass with a stride of the grid size, then waits at a grid barrier until every
// block has finished that pass (the next pass reads what all of them wrote).  The barrier
// is a counter the host clears before the launch; the wait is bounded (grid_wait), and a
// block that gives up records SP_ERR_TIMEOUT's cause in the plan's status word and leaves
// the kernel without running the remaining passes.  One block shape serves every pass:
// THREADS threads hold B = THREADS / T line columns (line passes) or THREADS / T_z pairs
// of real lines (z passes).
SP_D unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Arrive at barrier number `k` (1, 2, ...) of this launch and wait, at most `limit_ns`
// nanoseconds (and a bounded number of polls), until all `nblocks` blocks have arrived.
// Returns false, after setting *status, when the wait gave up.  All threads call it.
SP_D bool grid_wait(unsigned* count, int* status, unsigned k, unsigned nblocks, unsigned long long limit_ns)
{
    __shared__ int ok;
    __syncthreads();  // the block's writes of this pass precede the arrival
    if (threadIdx.x == 0) {
        ok = 1;
        __threadfence();
        atomicAdd(count, 1u);
        const unsigned target = k * nblocks;
        const unsigned long long t0 = global_ns();
        const unsigned long long max_polls = limit_ns / 16 + 1024;
        for (unsigned long long it = 0;; ++it) {
            const unsigned v = *(volatile unsigned*)count;
            if (v >= target) break;
            if (it >= max_polls || ((it & 31) == 0 && global_ns() - t0 > limit_ns)) {
                atomicExch(status, 1);
                ok = 0;
                break;
            }
            __nanosleep(128);
        }
        __threadfence();  // the other blocks' writes are visible after the wait
    }
    __syncthreads();
    return ok != 0;
}

struct PersistArgs {
    ZArgs2 z;           // z.B pairs per tile
    LArgs y, x;         // B columns per tile (compile-time in the kernel)
    int batch;
    int z_tiles, y_ncb, y_outer, x_ncb, x_outer;  // per right-hand side
    unsigned* bar;      // barrier counter, cleared before the launch
    int* status;
    unsigned long long limit_ns;
};

template <class R, int N> constexpr int persist_threads()
{
    constexpr int T = N / PlanOf<R, N>::E;
    return T * lanes_b_max<R, N>() < 256 ? T * lanes_b_max<R, N>() : 256;
}
template <class R, int N> constexpr int persist_lgb()
{
    constexpr int B = persist_threads<R, N>() / (N / PlanOf<R, N>::E);
    return B >= 16 ? 4 : (B >= 8 ? 3 : (B >= 4 ? 2 : (B >= 2 ? 1 : 0)));
}
template <class R, int N> constexpr int persist_bz() { return persist_threads<R, N>() / (N / PlanOf<ZKey<R>, N>::E); }
template <class R, int N> constexpr bool persist_ok()
{
    constexpr int TH = persist_threads<R, N>(), T = N / PlanOf<R, N>::E, Tz = N / PlanOf<ZKey<R>, N>::E;
    return TH % T == 0 && (1 << persist_lgb<R, N>()) * T == TH && TH % Tz == 0 && persist_bz<R, N>() >= 1 &&
           pairs_max<N>() % persist_bz<R, N>() == 0;
}
template <class R, int N> constexpr size_t persist_smem()
{
    constexpr int B = 1 << persist_lgb<R, N>();
    constexpr size_t lbuf = sizeof(cpx<R>) * (size_t)LayStrided<R>::size(N, B);
    constexpr size_t ltw = pass_tw_bytes<R, N>();
    constexpr size_t line = ltw + (two_buffers(lbuf, ltw) ? 2 : 1) * lbuf + stage_m_bytes<R, N, XMUL>(B);
    constexpr size_t zbuf = sizeof(cpx<R>) * (size_t)persist_bz<R, N>() * LayLine<N>::LD;
    constexpr size_t ztw = pass_tw_bytes<R, N, ZKey<R>>();
    constexpr size_t zs = ztw + (two_buffers(zbuf, ztw) ? 2 : 1) * zbuf;
    return line > zs ? line : zs;
}

template <class R, class Tio, int N>
__global__ void __launch_bounds__(persist_threads<R, N>(), 1) k_persist(PersistArgs pa)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int LGB = persist_lgb<R, N>();
    const unsigned nb = gridDim.x;
    // pass 1: z forward
    const int zt = pa.batch * pa.z_tiles;
    for (int tile = blockIdx.x; tile < zt; tile += gridDim.x) {
        zf_tile<R, Tio, N>(pa.z, tile % pa.z_tiles, tile / pa.z_tiles, smraw);
        __syncthreads();
    }
    if (!grid_wait(pa.bar, pa.status, 1, nb, pa.limit_ns)) return;
    // pass 2: y forward; pass 3: x forward * M * x inverse; pass 4: y inverse
    const int yt = pa.batch * pa.y_outer * pa.y_ncb;
    for (int tile = blockIdx.x; tile < yt; tile += gridDim.x) {
        const int r = tile / pa.y_ncb;
        line_tile<R, N, FWD, LGB>(pa.y, tile % pa.y_ncb, r % pa.y_outer, r / pa.y_outer, smraw);
        __syncthreads();
    }
    if (!grid_wait(pa.bar, pa.status, 2, nb, pa.limit_ns)) return;
    const int xt = pa.batch * pa.x_outer * pa.x_ncb;
    for (int tile = blockIdx.x; tile < xt; tile += gridDim.x) {
        const int r = tile / pa.x_ncb;
        line_tile<R, N, XMUL, LGB>(pa.x, tile % pa.x_ncb, r % pa.x_outer, r / pa.x_outer, smraw);
        __syncthreads();
    }
    if (!grid_wait(pa.bar, pa.status, 3, nb, pa.limit_ns)) return;
    for (int tile = blockIdx.x; tile < yt; tile += gridDim.x) {
        const int r = tile / pa.y_ncb;
        line_tile<R, N, INV, LGB>(pa.y, tile % pa.y_ncb, r % pa.y_outer, r / pa.y_outer, smraw);
        __syncthreads();
    }
    if (!grid_wait(pa.bar, pa.status, 4, nb, pa.limit_ns)) return;
    // pass 5: z inverse
    for (int tile = blockIdx.x; tile < zt; tile += gridDim.x) {
        zi_tile<R, Tio, N>(pa.z, tile % pa.z_tiles, tile / pa.z_tiles, smraw);
        __syncthreads();
    }
}

// Bounded wait of the persistent solve's barrier: a wait shorter than any pass would
// report a timeout for a healthy solve.
constexpr unsigned long long kPersistLimitNs = 2000000000ull;  // 2 s

template <class R, class Tio> struct PersistRun {
    sp_plan p;
    const void* rho;
    void* u;
    int batch;
    cudaStream_t st;
    template <int N> sp_status run()
    {
        if constexpr (!persist_ok<R, N>()) {
            return sp_fail(SP_ERR_UNSUPPORTED_SIZE, "no persistent solve for padded length %d in this precision", N);
        } else {
            constexpr int TH = persist_threads<R, N>(), B = 1 << persist_lgb<R, N>();
            constexpr size_t smem = persist_smem<R, N>();
            PersistArgs pa = {};
            ZArgs2& z = pa.z;
            z.rho = rho;
            z.u = u;
            z.W = p->d_work;
            z.n1 = p->n[1];
            z.n2 = p->n[2];
            z.lines = (long long)p->n[0] * p->n[1];
            z.plane = p->plane;
            z.ldz = p->ldz;
            z.io_bs = (long long)p->n[0] * p->n[1] * p->n[2];
            z.w_bs = (long long)p->n[0] * p->plane;
            z.tw = Tabs<R>::tw(p, 2);
            z.B = persist_bz<R, N>();
            LArgs& y = pa.y;
            y.in = y.out = p->d_work;
            y.in_os = y.out_os = p->plane;
            y.in_es = y.out_es = p->ldz;
            y.in_bs = y.out_bs = (long long)p->n[0] * p->plane;
            y.ncol = p->n[2] + 1;
            y.in_ld = p->ldz;
            y.tw = Tabs<R>::tw(p, 1);
            y.B = B;
            y.lgB = persist_lgb<R, N>();
            pa.x = y;
            LArgs& x = pa.x;
            x.in_os = x.out_os = p->ldz;
            x.in_es = x.out_es = p->plane;
            x.tw = Tabs<R>::tw(p, 0);
            x.M = Tabs<R>::M(p);
            x.No = p->N[1];
            x.nh_line = p->n[0];
            x.ldzM = p->ldz;
            pa.batch = batch;
            pa.z_tiles = (int)(((z.lines + 1) / 2 + z.B - 1) / z.B);
            pa.y_ncb = pa.x_ncb = (y.ncol + B - 1) / B;
            pa.y_outer = p->n[0];
            pa.x_outer = p->N[1];
            pa.bar = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(p->d_status) + 64);
            pa.status = p->d_status;
            pa.limit_ns = kPersistLimitNs;
            sp_status rc;
            if ((rc = smem_attr<k_persist<R, Tio, N>>(smem))) return rc;
            static std::atomic<int> per_sm_cached{0};
            int per_sm = per_sm_cached.load(std::memory_order_relaxed);
            if (!per_sm) {
                if ((rc = sp_cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist<R, Tio, N>, TH,
                                                                                      smem), "persistent occupancy")))
                    return rc;
                if (per_sm < 1) return sp_fail(SP_ERR_UNSUPPORTED_SIZE, "persistent solve: no block fits an SM");
                per_sm_cached.store(per_sm, std::memory_order_relaxed);
            }
            int dev = 0, sms = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const long long most = (long long)batch * (pa.x_outer * pa.x_ncb > 2 * pa.z_tiles ? pa.x_outer * pa.x_ncb : pa.z_tiles);
            const int nblocks = (int)(most < (long long)per_sm * sms ? most : (long long)per_sm * sms);
            if ((rc = sp_cuda_check(cudaMemsetAsync(pa.bar, 0, sizeof(unsigned), st), "clear grid barrier"))) return rc;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)nblocks);
            cfg.blockDim = dim3((unsigned)TH);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            return sp_cuda_check(cudaLaunchKernelEx(&cfg, k_persist<R, Tio, N>, pa), "persistent solve launch");
        }
    }
};

// The whole (batched) solve as one persistent cooperative launch, for cubic grids whose
// padded length has a compiled plan.
template <class R, class Tio>
sp_status solve_persistent(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st)
{
    if (!(p->N[0] == p->N[1] && p->N[1] == p->N[2]) || !len_ok(p->N[0]))
        return sp_fail(SP_ERR_UNSUPPORTED_SIZE, "the persistent solve needs a cubic grid with a compiled padded length");
    p->npass = 1;
    p->pass_name[0] = "persistent";
    sp_status rc;
    if ((rc = sp_mark(p, st))) return rc;
    if ((rc = with_len(p->N[0], PersistRun<R, Tio>{p, rho, u, batch, st}))) return rc;
    return sp_mark(p, st);
}

// Forward half only (diagnostic): spectrum[kx][ky][kz], kz <= n2 dense.
template <class R, class Tio>
sp_status forward(sp_plan p, const void* rho, void* spec, cudaStream_t st)
{
    for (int ax = 0; ax < 3; ++ax)
        if (!len_ok(p->N[ax])) return SP_ERR_UNSUPPORTED_SIZE;
    ZArgs2 z = {};
    z.rho = rho;
    z.W = p->d_work;
    z.n1 = p->n[1];
    z.n2 = p->n[2];
    z.lines = (long long)p->n[0] * p->n[1];
    z.plane = p->plane;
    z.ldz = p->ldz;
    z.tw = Tabs<R>::tw(p, 2);
    z.B = p->tile_z;
    LArgs y = {};
    y.in = y.out = p->d_work;
    y.in_os = y.out_os = p->plane;
    y.in_es = y.out_es = p->ldz;
    y.ncol = p->n[2] + 1;
    y.in_ld = p->ldz;
    y.tw = Tabs<R>::tw(p, 1);
    y.B = p->tile_line[1];
    LArgs x = y;
    x.B = p->tile_line[0];
    x.out = spec;
    x.in_os = p->ldz;
    x.in_es = p->plane;
    x.out_os = p->n[2] + 1;
    x.out_es = (long long)p->N[1] * (p->n[2] + 1);
    x.tw = Tabs<R>::tw(p, 0);
    sp_status rc;
    if ((rc = with_len(p->N[2], ZRun<R, Tio>{&z, true, 1, st}))) return rc;
    if ((rc = with_len(p->N[1], LineRun<R, FWD>{&y, p->n[0], 1, st, p->line_variant[1]}))) return rc;
    return with_len(p->N[0], LineRun<R, FWD>{&x, p->N[1], 1, st, p->line_variant[0]});
}

}  // namespace v2

// Explicit instantiation of the line-pass launchers for one arithmetic type R, so that
// they can be compiled in a translation unit of their own (PREFIX = extern to declare).
#define SP_V2_LINES_N(PREFIX, R, N)                                                          \
    PREFIX template sp_status v2::launch_line<R, N, v2::FWD>(const v2::LArgs&, int, int, cudaStream_t); \
    PREFIX template sp_status v2::launch_line<R, N, v2::INV>(const v2::LArgs&, int, int, cudaStream_t); \
    PREFIX template sp_status v2::launch_line<R, N, v2::XMUL>(const v2::LArgs&, int, int, cudaStream_t);
// The line-pass launchers of the alternative radix plan (AltPlan) of type R at length N.
#define SP_V2_ALT(PREFIX, R, N)                                                                   \
    PREFIX template sp_status v2::launch_line<R, N, v2::FWD, LineKey<R, 1>>(const v2::LArgs&, int, int,  \
                                                                             cudaStream_t);      \
    PREFIX template sp_status v2::launch_line<R, N, v2::INV, LineKey<R, 1>>(const v2::LArgs&, int, int,  \
                                                                             cudaStream_t);      \
    PREFIX template sp_status v2::launch_line<R, N, v2::XMUL, LineKey<R, 1>>(const v2::LArgs&, int, int, \
                                                                              cudaStream_t);
#define SP_V2_LINES(PREFIX, R)        \
    SP_V2_LINES_N(PREFIX, R, 64)      \
    SP_V2_LINES_N(PREFIX, R, 128)     \
    SP_V2_LINES_N(PREFIX, R, 192)     \
    SP_V2_LINES_N(PREFIX, R, 256)     \
    SP_V2_LINES_N(PREFIX, R, 384)     \
    SP_V2_LINES_N(PREFIX, R, 512)     \
    SP_V2_LINES_N(PREFIX, R, 1024)
