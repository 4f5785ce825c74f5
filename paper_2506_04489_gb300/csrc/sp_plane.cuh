// Fused plane passes of the FP32 solve (the three-pass schedule of Alg. 2): one kernel
// does the z real-to-complex transform and the y transform of an x-plane, another the y
// inverse and the z complex-to-real transform, so the z-transformed plane never goes
// through global memory.  Only the x pass (x forward * M * x inverse) stays a pass of
// its own.
//
// One x-plane is one thread-block cluster of C = 8 CTAs (distributed shared memory).
// Forward (plane_fwd):
//   phase Z : CTA r transforms the real rows y in [r RP, (r+1) RP) (RP = n1 / C), two rows
//             per complex transform, and writes each half spectrum X[y][kz] (kz <= n2)
//             into the shared memory of the CTA that owns column kz (CW = n2 / C columns
//             each, kz = r CW + c);
//   barrier : cluster-wide;
//   phase Y : CTA c transforms its CW columns along y (length 2 n1, rows y >= n1 zero)
//             and writes W[x][ky][kz] to global memory.
// Inverse (plane_inv): the same in reverse (y inverse keeping y < n1, scattered by row;
// then the z transforms of whole rows, cropped to z < n2).
// Columns kz = 0 and kz = n2 of a real row's half spectrum are real, so they travel as
// one complex column (kz = 0 in the real part, kz = n2 in the imaginary part): each CTA
// owns exactly CW columns.  Forward, the packed column's y transform P = Y0 + i Yn is
// split with Y0[k] = (P[k] + conj P[-k]) / 2, Yn[k] = (P[k] - conj P[-k]) / (2i); inverse,
// the two y-inverse results are real and are the real and imaginary parts.
// Included by the FP32 translation unit only.
#pragma once

#include <cooperative_groups.h>

#include "sp_v2.cuh"

namespace v2 {
namespace cg = cooperative_groups;

constexpr int kPlaneC = 8;        // CTAs per cluster (portable cluster size)
constexpr int kPlaneThreads = 512;

// The y phase's plan: eight values a thread (few registers, so 512 threads fit), the
// alternative plan of FP32 at this length, whose staged twiddles the plan already holds.
template <class R, int N> using PlaneYKey = LineKey<R, 1>;

// values a thread of the y phase's plan (1 where the plan does not exist: never used)
template <class R, int N> constexpr int plane_y_e()
{
    if constexpr (AltPlan<R, N>::exists) return PlanOf<PlaneYKey<R, N>, N>::E;
    else return 1;
}

template <class R, int N1, int N2> struct PlaneGeo {
    static constexpr int n1 = N1 / 2, n2 = N2 / 2;
    static constexpr int RP = n1 / kPlaneC;  // rows per CTA
    static constexpr int CW = n2 / kPlaneC;  // columns per CTA
    static constexpr int Tz = N2 / PlanOf<ZKey<R>, N2>::E;
    static constexpr int BZ = kPlaneThreads / Tz;  // pairs of rows per z round
    static constexpr int Ty = N1 / plane_y_e<R, N1>();
    static constexpr int BY = kPlaneThreads / Ty;  // columns per y chunk
    static constexpr int LGBY = BY >= 16 ? 4 : (BY >= 8 ? 3 : (BY >= 4 ? 2 : (BY >= 2 ? 1 : 0)));
    // shared memory: the stage (RP x n2 or n1 x CW complex), then one exchange buffer for
    // the z phase or the y phase, then N1 complex of scratch for the packed column
    static constexpr int STAGE = (n1 * CW > RP * n2 ? n1 * CW : RP * n2);
    static constexpr int ZBUF = BZ * LayLine<N2>::LD;
    static constexpr int YBUF = LayStrided<R>::size(N1, BY);
    static constexpr int BUF = ZBUF > YBUF ? ZBUF : YBUF;
    static constexpr size_t smem = sizeof(cpx<R>) * (size_t)(STAGE + BUF + N1);
    static constexpr bool ok = AltPlan<R, N1>::exists && tw_global<R, N1>() && tw_global<R, N2>() && n1 % (2 * kPlaneC) == 0 &&
                               n2 % kPlaneC == 0 && (RP / 2) % BZ == 0 && CW % BY == 0 && (1 << LGBY) == BY &&
                               BZ * Tz == kPlaneThreads && BY * Ty == kPlaneThreads && smem <= 227 * 1024;
};

struct PlaneArgs {
    const void* rho;  // forward input / inverse output (u), [b][x][y][z]
    void* u;
    void* W;          // workspace, [b][x][ky][kz], row stride ldz
    const void* twz;  // z-axis twiddles (base N2 entries, then the staged tables)
    const void* twy;  // y-axis twiddles
    long long plane, io_bs, w_bs;
    int ldz;
};

template <class R, class Tio, int N1, int N2>
__global__ void __launch_bounds__(kPlaneThreads, 2) k_plane_fwd(PlaneArgs a)
{
    using G = PlaneGeo<R, N1, N2>;
    using KZ = ZKey<R>;
    using KY = PlaneYKey<R, N1>;
    constexpr int n1 = G::n1, n2 = G::n2, RP = G::RP, CW = G::CW, Tz = G::Tz, BZ = G::BZ, BY = G::BY;
    constexpr int EZ = PlanOf<KZ, N2>::E, R0Z = PlanOf<KZ, N2>::R[0];
    constexpr int EY = PlanOf<KY, N1>::E, R0Y = PlanOf<KY, N1>::R[0];
    cg::cluster_group cluster = cg::this_cluster();
    const int r = (int)cluster.block_rank();
    const int x = blockIdx.x / kPlaneC, batch = blockIdx.y;
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<R>* stage = reinterpret_cast<cpx<R>*>(smraw);       // [y < n1][c < CW]
    cpx<R>* buf = stage + G::STAGE;
    cpx<R>* scratch = buf + G::BUF;                          // N1 entries
    const int tid = threadIdx.x;
    const Tio* rho = static_cast<const Tio*>(a.rho) + batch * a.io_bs + (long long)x * n1 * n2;
    cpx<R>* W = static_cast<cpx<R>*>(a.W) + batch * a.w_bs + (long long)x * a.plane;
    // ---- phase Z: rows y in [r RP, (r+1) RP), BZ pairs a round
    {
        const cpx<R>* tws = static_cast<const cpx<R>*>(a.twz) + N2;
        const int pb = tid / Tz, t = tid % Tz;
        const LayLine<N2> lay{pb * LayLine<N2>::LD};
        for (int round = 0; round < RP / 2 / BZ; ++round) {
            const int y0 = r * RP + 2 * (round * BZ + pb), y1 = y0 + 1;
            cpx<R> v[EZ];
#pragma unroll
            for (int j = 0; j < EZ; ++j) {
                const int z = first_element<KZ, N2, false>(t, j);
                R xr = Num<R>::c(0.0), xi = Num<R>::c(0.0);
                if ((j % R0Z) < R0Z / 2) {  // z < n2: the padded half is zero
                    xr = to_r<R, Tio>(rho[(long long)y0 * n2 + z]);
                    xi = to_r<R, Tio>(rho[(long long)y1 * n2 + z]);
                }
                v[j] = mk(xr, xi);
            }
            cpx<R>* sm = run_stages<R, N2, false, -1, true, KZ>(v, buf, buf, lay, tws, t);
#pragma unroll
            for (int j = 0; j < EZ; ++j) sm[lay(last_element<KZ, N2, false>(t, j))] = v[j];
            __syncthreads();
            // two real rows from one complex transform; each value goes to its column's
            // owner (columns 0 and n2 packed into column 0: both are real)
            for (int k = t; k <= n2; k += Tz) {
                const cpx<R> zk = sm[lay(k)];
                const cpx<R> zm = conjg(sm[lay(k == 0 ? 0 : N2 - k)]);
                const cpx<R> s = zk + zm, d = zk - zm;
                const cpx<R> xa = half_of(s), xb = half_of(mk(im_of(d), -re_of(d)));
                if (k > 0 && k < n2) {
                    cpx<R>* dst = cluster.map_shared_rank(stage, k / CW);
                    dst[y0 * CW + k % CW] = xa;
                    dst[y1 * CW + k % CW] = xb;
                } else {
                    R* dst = reinterpret_cast<R*>(cluster.map_shared_rank(stage, 0));
                    const int part = k == 0 ? 0 : 1;  // real part: kz = 0, imaginary part: kz = n2
                    dst[2 * (y0 * CW) + part] = re_of(xa);
                    dst[2 * (y1 * CW) + part] = re_of(xb);
                }
            }
            __syncthreads();  // the exchange buffer is rewritten next round
        }
    }
    cluster.sync();  // every CTA's columns are complete
    // ---- phase Y: my columns kz = r CW + c, BY at a time
    {
        const cpx<R>* tws = static_cast<const cpx<R>*>(a.twy) + N1 + tw_key_offset<R, N1, KY>();
        const int b = tid & (BY - 1), t = tid >> G::LGBY;
        const LayStrided<R> lay(G::LGBY, b);
        for (int ch = 0; ch < CW / BY; ++ch) {
            const int c = ch * BY + b;
            const bool packed = r == 0 && c == 0;
            cpx<R> v[EY];
#pragma unroll
            for (int j = 0; j < EY; ++j) {
                const int y = first_element<KY, N1, false>(t, j);
                v[j] = ((j % R0Y) < R0Y / 2) ? stage[y * CW + c] : czero<R>();
            }
            __syncthreads();  // buf is free (previous chunk's reads, or the z phase)
            run_stages<R, N1, false, -1, true, KY>(v, buf, buf, lay, tws, t);
            const int kz = r * CW + c;
            if (r == 0 && ch == 0) {  // the packed column: split P = Y0 + i Yn through scratch
                if (b == 0) {
#pragma unroll
                    for (int j = 0; j < EY; ++j) scratch[last_element<KY, N1, false>(t, j)] = v[j];
                }
                __syncthreads();
            }
#pragma unroll
            for (int j = 0; j < EY; ++j) {
                const int ky = last_element<KY, N1, false>(t, j);
                if (!packed) {
                    W[(long long)ky * a.ldz + kz] = v[j];
                } else {
                    const cpx<R> p = v[j], q = conjg(scratch[ky == 0 ? 0 : N1 - ky]);
                    const cpx<R> s = p + q, d = p - q;
                    W[(long long)ky * a.ldz] = half_of(s);
                    W[(long long)ky * a.ldz + n2] = half_of(mk(im_of(d), -re_of(d)));
                }
            }
        }
    }
}

template <class R, class Tio, int N1, int N2>
__global__ void __launch_bounds__(kPlaneThreads, 2) k_plane_inv(PlaneArgs a)
{
    using G = PlaneGeo<R, N1, N2>;
    using KZ = ZKey<R>;
    using KY = PlaneYKey<R, N1>;
    constexpr int n1 = G::n1, n2 = G::n2, RP = G::RP, CW = G::CW, Tz = G::Tz, BZ = G::BZ, BY = G::BY;
    constexpr int EZ = PlanOf<KZ, N2>::E, R0Z = PlanOf<KZ, N2>::R[0];
    constexpr int EY = PlanOf<KY, N1>::E, R0Y = PlanOf<KY, N1>::R[0];
    cg::cluster_group cluster = cg::this_cluster();
    const int r = (int)cluster.block_rank();
    const int x = blockIdx.x / kPlaneC, batch = blockIdx.y;
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<R>* stage = reinterpret_cast<cpx<R>*>(smraw);  // [y < RP][kz < n2], kz = 0 packed
    cpx<R>* buf = stage + G::STAGE;
    const int tid = threadIdx.x;
    Tio* u = static_cast<Tio*>(a.u) + batch * a.io_bs + (long long)x * n1 * n2;
    const cpx<R>* W = static_cast<const cpx<R>*>(a.W) + batch * a.w_bs + (long long)x * a.plane;
    // ---- phase Y: my columns, y inverse (all 2 n1 rows in), keep y < n1, scatter by row
    {
        const cpx<R>* tws = static_cast<const cpx<R>*>(a.twy) + N1 + tw_key_offset<R, N1, KY>();
        const int b = tid & (BY - 1), t = tid >> G::LGBY;
        const LayStrided<R> lay(G::LGBY, b);
        for (int ch = 0; ch < CW / BY; ++ch) {
            const int c = ch * BY + b, kz = r * CW + c;
            const bool packed = r == 0 && c == 0;
            cpx<R> v[EY];
#pragma unroll
            for (int j = 0; j < EY; ++j) {
                const int ky = first_element<KY, N1, true>(t, j);
                const cpx<R> w0 = W[(long long)ky * a.ldz + kz];
                if (packed) {  // P = W[.][0] + i W[.][n2]
                    const cpx<R> wn = W[(long long)ky * a.ldz + n2];
                    v[j] = mk(re_of(w0) - im_of(wn), im_of(w0) + re_of(wn));
                } else {
                    v[j] = w0;
                }
            }
            __syncthreads();  // buf is free
            run_stages<R, N1, true, +1, false, KY>(v, buf, buf, lay, tws, t);
#pragma unroll
            for (int j = 0; j < EY; ++j) {
                if ((j % R0Y) < R0Y / 2) {  // y < n1
                    const int y = last_element<KY, N1, true>(t, j);
                    cpx<R>* dst = cluster.map_shared_rank(stage, y / RP);
                    dst[(y % RP) * n2 + kz] = v[j];  // packed: (column 0, column n2) as (re, im)
                }
            }
        }
    }
    cluster.sync();
    // ---- phase Z: my rows, two per complex transform, cropped to z < n2
    {
        const cpx<R>* tws = static_cast<const cpx<R>*>(a.twz) + N2;
        const int pb = tid / Tz, t = tid % Tz;
        const LayLine<N2> lay{pb * LayLine<N2>::LD};
        for (int round = 0; round < RP / 2 / BZ; ++round) {
            const int ly0 = 2 * (round * BZ + pb), ly1 = ly0 + 1;  // local rows
            __syncthreads();  // buf is free (y phase or previous round)
            // Z_k = Xa_k + i Xb_k from the Hermitian halves (DC and Nyquist real)
            for (int k = t; k <= n2; k += Tz) {
                R ar, ai, br, bi;
                if (k == 0 || k == n2) {
                    const cpx<R> pa = stage[ly0 * n2], pbk = stage[ly1 * n2];
                    ar = k == 0 ? re_of(pa) : im_of(pa);
                    br = k == 0 ? re_of(pbk) : im_of(pbk);
                    ai = bi = Num<R>::c(0.0);
                } else {
                    const cpx<R> xa = stage[ly0 * n2 + k], xb = stage[ly1 * n2 + k];
                    ar = re_of(xa);
                    ai = im_of(xa);
                    br = re_of(xb);
                    bi = im_of(xb);
                }
                buf[lay(k)] = mk(ar - bi, ai + br);
                if (k > 0 && k < n2) buf[lay(N2 - k)] = mk(ar + bi, br - ai);
            }
            __syncthreads();
            cpx<R> v[EZ];
            Stage<R, N2, true, 0, KZ>::load(v, buf, lay, t);
            __syncthreads();  // one buffer: every load precedes the first stage's writes
            run_stages<R, N2, true, +1, false, KZ>(v, buf, buf, lay, tws, t);
            const int y0 = r * RP + ly0, y1 = y0 + 1;
#pragma unroll
            for (int j = 0; j < EZ; ++j) {
                if ((j % R0Z) < R0Z / 2) {  // z < n2
                    const int z = last_element<KZ, N2, true>(t, j);
                    u[(long long)y0 * n2 + z] = from_r<R, Tio>(re_of(v[j]));
                    u[(long long)y1 * n2 + z] = from_r<R, Tio>(im_of(v[j]));
                }
            }
        }
    }
}

template <class R, class Tio> struct PlaneRun {
    sp_plan p;
    PlaneArgs a;
    int batch;
    bool forward;
    cudaStream_t st;
    template <int N> sp_status run()
    {
        if constexpr (!PlaneGeo<R, N, N>::ok) {
            return sp_fail(SP_ERR_UNSUPPORTED_SIZE, "no fused plane pass for padded length %d", N);
        } else {
            using G = PlaneGeo<R, N, N>;
            sp_status rc;
            if (forward) {
                if ((rc = smem_attr<k_plane_fwd<R, Tio, N, N>>(G::smem))) return rc;
            } else {
                if ((rc = smem_attr<k_plane_inv<R, Tio, N, N>>(G::smem))) return rc;
            }
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)(p->n[0] * kPlaneC), (unsigned)batch);
            cfg.blockDim = dim3(kPlaneThreads);
            cfg.dynamicSmemBytes = G::smem;
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = kPlaneC;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            const cudaError_t e = forward ? cudaLaunchKernelEx(&cfg, k_plane_fwd<R, Tio, N, N>, a)
                                          : cudaLaunchKernelEx(&cfg, k_plane_inv<R, Tio, N, N>, a);
            return sp_cuda_check(e, forward ? "fused plane pass (forward)" : "fused plane pass (inverse)");
        }
    }
};

template <class R> struct PlaneOk {
    template <int N> sp_status run() { return PlaneGeo<R, N, N>::ok ? SP_OK : SP_ERR_UNSUPPORTED_SIZE; }
};
// Whether the fused plane passes exist for this plan (same padded length on y and z).
template <class R> bool plane_supported(sp_plan p)
{
    return p->N[1] == p->N[2] && with_len(p->N[1], PlaneOk<R>{}) == SP_OK;
}

// The three-pass solve: fused forward plane pass, x pass, fused inverse plane pass.
template <class R, class Tio>
sp_status solve_fused(sp_plan p, const void* rho, void* u, int batch, cudaStream_t st, bool mark)
{
    for (int ax = 0; ax < 3; ++ax)
        if (!len_ok(p->N[ax])) return SP_ERR_UNSUPPORTED_SIZE;
    if (!plane_supported<R>(p)) return sp_fail(SP_ERR_UNSUPPORTED_SIZE, "no fused plane passes for this grid");
    sp_status rc;
    p->npass = 3;
    p->pass_name[0] = "plane_forward";
    p->pass_name[1] = "x_multiply";
    p->pass_name[2] = "plane_inverse";
    PlaneArgs pa;
    pa.rho = rho;
    pa.u = u;
    pa.W = p->d_work;
    pa.twz = Tabs<R>::tw(p, 2);
    pa.twy = Tabs<R>::tw(p, 1);
    pa.plane = p->plane;
    pa.io_bs = (long long)p->n[0] * p->n[1] * p->n[2];
    pa.w_bs = (long long)p->n[0] * p->plane;
    pa.ldz = p->ldz;
    LArgs x = {};
    x.in = x.out = p->d_work;
    x.in_os = x.out_os = p->ldz;
    x.in_es = x.out_es = p->plane;
    x.in_bs = x.out_bs = (long long)p->n[0] * p->plane;
    x.ncol = p->n[2] + 1;
    x.in_ld = p->ldz;
    x.tw = Tabs<R>::tw(p, 0);
    x.M = Tabs<R>::M(p);
    x.B = p->tile_line[0];
    x.No = p->N[1];
    x.nh_line = p->n[0];
    x.ldzM = p->ldz;
    if (mark && (rc = sp_mark(p, st))) return rc;
    if ((rc = with_len(p->N[1], PlaneRun<R, Tio>{p, pa, batch, true, st}))) return rc;
    if (mark && (rc = sp_mark(p, st))) return rc;
    if ((rc = with_len(p->N[0], LineRun<R, XMUL>{&x, p->N[1], batch, st, p->line_variant[0]}))) return rc;
    if (mark && (rc = sp_mark(p, st))) return rc;
    if ((rc = with_len(p->N[1], PlaneRun<R, Tio>{p, pa, batch, false, st}))) return rc;
    if (mark && (rc = sp_mark(p, st))) return rc;
    return SP_OK;
}

}  // namespace v2
