// diffusion2d_tb.cu -- K forward-Euler steps of the 2D heat equation per pass over the field
// (Sec. 3.2, Eqs. 4-7 in 2D, radius r = 1..4 of Sec. 5.3), FP32, periodic boundaries: temporal
// blocking.
//
// f_{s} = g0 f_{s-1} + sum_{axis in x,y} sum_{a=1..R} g_{axis,a} (f_{s-1}(+a) + f_{s-1}(-a)),
// s = 1..K, so one pass reads f_0 once and writes f_K once instead of K reads and K writes.
//
// GB300 design: one warp streams one vertical strip of the domain.
//   * The strip's output is TX = 4 TXG cells wide.  Stage s (the s-th step) is computed on the
//     strip widened by (K - s) R cells per side (rounded out to whole float4 groups), so stage 1
//     spans exactly 32 groups, one per lane, and stage K is the strip itself.  The widening
//     (K - 1) R cells per side is the only redundant work: about 10 % at r = 3, K = 4.
//   * Rows stream in y.  A new row of f_0 enters per iteration, and stage s then computes its
//     row lagging s R rows behind.  Each lane keeps, per stage, a register queue of the 2R+1
//     input rows at its own group (y neighbours come from registers); x neighbours come from
//     the stage's input row in a small per-warp shared-memory ring.  A cell therefore costs one
//     16-byte store and three 16-byte loads of shared memory per stage, the bound being shared
//     memory bandwidth.  Stage K's row goes to global memory with its periodic images (Eq. 2).
//   * f_0 rows are fetched with 16-byte cp.async copies, P rows ahead, from periodically wrapped
//     coordinates: the widened strip at a face reads the far side of the domain directly, so
//     the kernel needs no halo in its input at all (nx a multiple of 4, so no float4 group
//     straddles the wrap).
//   * The warps of a CTA work on independent strips and synchronise only within the warp.
//   * A strip is split into row chunks so that the grid fills the SMs.  Each chunk re-reads 2KR
//     rows of f_0 (from L2) and recomputes the widened stages on them.
// The multiply-add order per cell is x, y for a = 1 .. R, as in the other heat kernels.
#include <algorithm>
#include <utility>

#include "internal.h"

namespace stn {
namespace {

constexpr int TB_WARPS = 4;  // warps (independent strips) per CTA

// Extra float4 groups per side of stage s's row (s = 0 .. K; stage 0 is f_0, which stage 1
// reads R cells beyond its own width).
__host__ __device__ constexpr int tb_g(int K, int s, int R) { return s == 0 ? tb_g(K, 1, R) + 1 : ((K - s) * R + 3) / 4; }

// Slot of row index v in a ring of n rows (for any integer v).
__host__ __device__ constexpr int tb_slot(int v, int n) { return ((v % n) + n) % n; }

template <int R, int K> struct Tb {
    static constexpr int G0 = tb_g(K, 0, R);
    static constexpr int G1 = tb_g(K, 1, R);
    static constexpr int TXG = 32 - 2 * G1;  // output groups per strip
    static constexpr int TX = 4 * TXG;       // output cells per strip
    static constexpr int W = TXG + 2 * G0;   // groups per ring row (stage 0 width)
    static constexpr int NQ = 2 * R + 1;     // register queue rows per stage
    // The row loop is unrolled over NL = 2 NQ iterations, so every queue entry and ring slot is a
    // compile-time constant.  The f_0 ring has NL rows and runs P rows ahead (its oldest row in
    // use lags R behind the newest); the rings of stages 1 .. K-1 have NQ rows.
    static constexpr int NL = 2 * NQ;
    static constexpr int P = (3 * R + 1) < 7 ? (3 * R + 1) : 7;
    static constexpr int RING0 = NL * W * 4;  // floats
    static constexpr int RINGI = NQ * W * 4;
    static constexpr int WARP_FLOATS = RING0 + (K - 1) * RINGI;
    static constexpr size_t SMEM = (size_t)TB_WARPS * WARP_FLOATS * sizeof(float);
    static_assert(R >= 1 && R <= 4, "radius 1..4: one float4 group per side covers the x neighbours");
    static_assert(TXG >= 8, "strip too narrow");
    static_assert(W <= 64, "two groups per lane at most");
    static_assert(P + R < NL, "the f_0 ring holds the prefetched rows and the R rows in use");
};

struct W2f {  // folded weights
    float g0, gx[4], gy[4];
};

__device__ __forceinline__ void cp_async16(float *smem, const float *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// Ring row (float offset) of row index v in the input ring of stage S (ring 0 = f_0).
template <int R, int K, int S> __device__ __forceinline__ constexpr int tb_in_row(int v) {
    using C = Tb<R, K>;
    if constexpr (S == 1) return tb_slot(v, C::NL) * C::W * 4;
    else return C::RING0 + (S - 2) * C::RINGI + tb_slot(v, C::NQ) * C::W * 4;
}

// Stage S (1..K) at loop iteration j (j = U mod NL) for this lane's group:
//  1. the leading input row L = j - (S-1) R (just produced by stage S-1, or fetched for S = 1)
//     enters the lane's queue;
//  2. output row o = j - S R is computed from the queue (y neighbours, centre) and the x
//     neighbours of input row o in the ring, into ring S (S < K) or global memory (S == K).
template <int R, int K, int S, int U>
__device__ __forceinline__ void tb_stage(int lane, int j, int rows_in, float *rings, float4 (&Q)[2 * R + 1],
                                         float *__restrict__ out, const Geom &g, const W2f &w, int x0, int ys) {
    using C = Tb<R, K>;
    constexpr int GS = tb_g(K, S, R);
    if (lane >= C::TXG + 2 * GS) return;
    const int q = lane - GS + C::G0;  // ring slot of this lane's group
    const int L = j - (S - 1) * R;
    if (L >= (S - 1) * R && L < rows_in - (S - 1) * R)  // valid row of stage S-1 (warp-uniform)
        Q[tb_slot(U - (S - 1) * R, C::NQ)] = ld4(rings + tb_in_row<R, K, S>(U - (S - 1) * R) + 4 * q);
    const int o = j - S * R;
    if (o < S * R || o >= rows_in - S * R) return;  // row outside stage S's valid range
    constexpr int OC = U - S * R;  // o, before the mod
    const float *rc = rings + tb_in_row<R, K, S>(OC) + 4 * q;
    const float4 cl = ld4(rc - 4), cc = Q[tb_slot(OC, C::NQ)], cr = ld4(rc + 4);
    const float E[12] = {cl.x, cl.y, cl.z, cl.w, cc.x, cc.y, cc.z, cc.w, cr.x, cr.y, cr.z, cr.w};
    const float2 G0v = make_float2(w.g0, w.g0);
    float2 acc[2] = {__fmul2_rn(G0v, make_float2(E[4], E[5])), __fmul2_rn(G0v, make_float2(E[6], E[7]))};
#pragma unroll
    for (int a = 1; a <= R; ++a) {
        const float4 yp = Q[tb_slot(OC + a, C::NQ)], ym = Q[tb_slot(OC - a, C::NQ)];
        const float2 GX = make_float2(w.gx[a - 1], w.gx[a - 1]), GY = make_float2(w.gy[a - 1], w.gy[a - 1]);
        const float2 ys2[2] = {__fadd2_rn(make_float2(yp.x, yp.y), make_float2(ym.x, ym.y)),
                               __fadd2_rn(make_float2(yp.z, yp.w), make_float2(ym.z, ym.w))};
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int i0 = 4 + 2 * p;
            const float2 sx = (a % 2 == 0) ? __fadd2_rn(make_float2(E[i0 + a], E[i0 + 1 + a]),
                                                        make_float2(E[i0 - a], E[i0 + 1 - a]))
                                           : make_float2(E[i0 + a] + E[i0 - a], E[i0 + 1 + a] + E[i0 + 1 - a]);
            acc[p] = __ffma2_rn(GX, sx, acc[p]);
            acc[p] = __ffma2_rn(GY, ys2[p], acc[p]);
        }
    }
    const float4 res = make_float4(acc[0].x, acc[0].y, acc[1].x, acc[1].y);
    if constexpr (S < K) {
        *reinterpret_cast<float4 *>(rings + C::RING0 + (S - 1) * C::RINGI + tb_slot(OC, C::NQ) * C::W * 4 + 4 * q) =
            res;
    } else {
        const int nx = (int)g.n[0], ny = (int)g.n[1];
        const int x = x0 + 4 * (q - C::G0), y = ys - K * R + o;
        if (x >= nx) return;  // the last strip overhangs the domain
        if (x >= R && x + 4 <= nx - R && y >= R && y < ny - R) {
            *reinterpret_cast<float4 *>(out + g.idx(x, y, 0)) = res;
        } else {
            const float v[4] = {res.x, res.y, res.z, res.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) store_with_images(out, g, R, true, x + u, y, 0, v[u]);
        }
    }
}

template <int R, int K> struct TbQueues {
    float4 q[K][2 * R + 1];
};

template <int R, int K, int S, int U>
__device__ __forceinline__ void tb_stages(int lane, int j, int rows_in, float *rings, TbQueues<R, K> &qs, float *out,
                                          const Geom &g, const W2f &w, int x0, int ys) {
    tb_stage<R, K, S, U>(lane, j, rows_in, rings, qs.q[S - 1], out, g, w, x0, ys);
    __syncwarp();
    if constexpr (S < K) tb_stages<R, K, S + 1, U>(lane, j, rows_in, rings, qs, out, g, w, x0, ys);
}

// Per-lane state of the f_0 stream: the wrapped x offsets of the lane's (up to two) groups and
// the next row to fetch (wrapped in y).
struct TbStream {
    const float *in;
    int xoff[2];
    int ngroups;
    int yl;       // wrapped row index of the next f_0 row to fetch
    int64_t pitch;
    int64_t base;  // element index of (x = 0, y = 0)
};

template <int R, int K>
__device__ __forceinline__ void tb_issue(TbStream &st, float *ring0, int slot, int lane, int ny) {
    using C = Tb<R, K>;
    const float *src = st.in + st.base + (int64_t)st.yl * st.pitch;
    float *dst = ring0 + slot * C::W * 4 + 4 * lane;  // ring 0 (f_0) starts the warp's rings
    cp_async16(dst, src + st.xoff[0]);
    if (st.ngroups > 1) cp_async16(dst + 4 * 32, src + st.xoff[1]);
    st.yl = st.yl + 1 == ny ? 0 : st.yl + 1;
}

// One loop iteration j (j = U mod NL): fetch f_0 row j + P, wait for row j, run the K stages.
template <int R, int K, int U>
__device__ __forceinline__ void tb_iter(int lane, int j, int rows_in, float *rings, TbQueues<R, K> &qs, float *out,
                                        const Geom &g, const W2f &w, int x0, int ys, TbStream &st) {
    using C = Tb<R, K>;
    if (j >= rows_in) return;
    // the slot of row j + P held row j + P - NL < j - R, which stage 1 no longer reads
    if (j + C::P < rows_in) tb_issue<R, K>(st, rings, tb_slot(U + C::P, C::NL), lane, (int)g.n[1]);
    cp_async_commit();
    cp_async_wait<C::P>();  // row j has landed (this lane's copies) ...
    __syncwarp();           // ... and every lane's
    tb_stages<R, K, 1, U>(lane, j, rows_in, rings, qs, out, g, w, x0, ys);
}

template <int R, int K, int... Us>
__device__ __forceinline__ void tb_period(int lane, int j0, int rows_in, float *rings, TbQueues<R, K> &qs, float *out,
                                          const Geom &g, const W2f &w, int x0, int ys, TbStream &st,
                                          std::integer_sequence<int, Us...>) {
    (tb_iter<R, K, Us>(lane, j0 + Us, rows_in, rings, qs, out, g, w, x0, ys, st), ...);
}

template <int R, int K>
__global__ void __launch_bounds__(32 * TB_WARPS)
heat2d_tb_kernel(const float *__restrict__ in, float *__restrict__ out, Geom g, W2f w, int strips, int chunk_rows) {
    using C = Tb<R, K>;
    extern __shared__ __align__(16) float tb_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gw = blockIdx.x * TB_WARPS + wid;
    const int strip = gw % strips, chunk = gw / strips;
    const int nx = (int)g.n[0], ny = (int)g.n[1];
    const int ys = chunk * chunk_rows;
    pdl_launch_dependents();
    if (ys >= ny) return;  // whole warp: no block-level synchronisation follows
    const int count = min(chunk_rows, ny - ys);
    const int rows_in = count + 2 * K * R;
    const int x0 = strip * C::TX;
    float *rings = tb_smem + wid * C::WARP_FLOATS;  // ring 0: f_0; ring s: stage s
    TbQueues<R, K> qs;

    TbStream st;
    st.in = in;
    st.pitch = g.pad[0];
    st.base = g.idx(0, 0, 0);
    st.ngroups = lane + 32 < C::W ? 2 : 1;
#pragma unroll
    for (int h = 0; h < 2; ++h) {  // wrapped x of the lane's groups q = lane, lane + 32
        int x = (x0 + 4 * (lane + 32 * h - C::G0)) % nx;
        st.xoff[h] = x < 0 ? x + nx : x;
    }
    st.yl = (ys - K * R) % ny;
    if (st.yl < 0) st.yl += ny;
    pdl_wait();  // the input is the previous pass's output

#pragma unroll
    for (int j = 0; j < C::P; ++j) {
        if (j < rows_in) tb_issue<R, K>(st, rings, j, lane, ny);
        cp_async_commit();
    }
    for (int j0 = 0; j0 < rows_in; j0 += C::NL)
        tb_period<R, K>(lane, j0, rows_in, rings, qs, out, g, w, x0, ys, st, std::make_integer_sequence<int, C::NL>{});
}

template <int R, int K>
cudaError_t run_tb(const void *in, void *out, const Geom &g, const DiffCoef &dc, cudaStream_t s) {
    using C = Tb<R, K>;
    auto k = heat2d_tb_kernel<R, K>;
    static int occ[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64) return cudaErrorInvalidDevice;
    if (!occ[dev]) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, 32 * TB_WARPS, C::SMEM);
        if (e != cudaSuccess) return e;
        occ[dev] = std::max(o, 1);
    }
    W2f w;
    w.g0 = (float)dc.g0;
    for (int a = 0; a < 4; ++a) {
        w.gx[a] = (float)dc.ga[0][a];
        w.gy[a] = (float)dc.ga[1][a];
    }
    const int nx = (int)g.n[0], ny = (int)g.n[1];
    const int strips = (nx + C::TX - 1) / C::TX;
    // one wave of warps, but chunks of at least 8 KR rows so the 2KR re-read rows stay a
    // small fraction of each chunk
    const long resident = (long)occ[dev] * TB_WARPS * device_sms();
    int chunks = (int)std::max(1L, (resident + strips - 1) / strips);
    chunks = std::min(chunks, std::max(1, ny / (8 * K * R)));
    const int chunk_rows = (ny + chunks - 1) / chunks;
    chunks = (ny + chunk_rows - 1) / chunk_rows;
    const long warps = (long)strips * chunks;
    const unsigned blocks = (unsigned)((warps + TB_WARPS - 1) / TB_WARPS);
    return launch_pdl(k, dim3(blocks), dim3(32 * TB_WARPS), C::SMEM, s, static_cast<const float *>(in),
                      static_cast<float *>(out), g, w, strips, chunk_rows);
}

template <int K>
cudaError_t run_tb_r(const void *in, void *out, const Geom &g, const DiffCoef &c, cudaStream_t s) {
    switch (c.r) {
    case 1: return run_tb<1, K>(in, out, g, c, s);
    case 2: return run_tb<2, K>(in, out, g, c, s);
    case 3: return run_tb<3, K>(in, out, g, c, s);
    case 4: return run_tb<4, K>(in, out, g, c, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool diffusion2d_tb_ok(int dtype, const Geom &g) { return dtype == 2 && g.n[0] % 4 == 0; }

cudaError_t launch_diffusion2d_tb(int dtype, int steps, const void *in, void *out, const Geom &g, const DiffCoef &c,
                                  cudaStream_t s) {
    if (!diffusion2d_tb_ok(dtype, g)) return cudaErrorInvalidValue;
    if (steps == 2) return run_tb_r<2>(in, out, g, c, s);
    if (steps == 4) return run_tb_r<4>(in, out, g, c, s);
    return cudaErrorInvalidValue;
}

}  // namespace stn
