// diffusion.cu -- forward-Euler step of df/dt = alpha lap f (Sec. 3.2, Eqs. 4-7) in 3D.
//
// The Euler update and the three axis Laplacians fold into one 19-point cross-correlation
// (Eqs. 5 and 7): f' = g0 f + sum_axes sum_{a=1..3} g_{axis,a} (f(+a) + f(-a)).
//
// GB300 design (2.5D z-streaming):
//   * A CTA owns a TX x (BY*RY) tile of the xy-plane and marches along z over a chunk of ZC
//     planes.  Each padded input plane tile (TX + 2 HX) x (BY*RY + 6) is brought into a
//     ring of NSLOT shared-memory slots by one TMA load (cp.async.bulk.tensor.3d) signalled
//     on a per-slot mbarrier; loads run NSLOT - 3 planes ahead of the compute.
//   * Each thread keeps the z-column of its RY cells for planes z-3..z+3 in a register queue,
//     so z-neighbours cost no shared-memory traffic; x- and y-neighbours are read from the
//     centre plane in shared memory (conflict-free: a warp reads 32 consecutive words).
//   * Outputs are stored once, coalesced, and cells within r of a face also store their
//     periodic images (Eq. 2), so the next step needs no separate halo pass.
//   * Waits are bounded (globaltimer); on expiry the CTA records ERR_TIMEOUT, drains its
//     in-flight TMA loads (again bounded) and returns.
#include "internal.h"

namespace stn {

template <typename T> struct DC {
    T g0;
    T ga[3][3];
};

template <typename T, int TX, int BY, int RY, int NSLOT, int ZC>
struct DiffCfg {
    static constexpr int HX = 16 / sizeof(T) >= 4 ? 16 / (int)sizeof(T) : 4;  // 4 for f32/f64
    static constexpr int TY = BY * RY;
    static constexpr int TXP = TX + 2 * HX;
    static constexpr int ROWS = TY + 2 * R6;
    static constexpr int SLOT_ELEMS = ((TXP * ROWS * (int)sizeof(T) + 127) / 128) * 128 / (int)sizeof(T);
    static constexpr uint32_t BOX_BYTES = TXP * ROWS * sizeof(T);
    static constexpr size_t SMEM = (size_t)NSLOT * SLOT_ELEMS * sizeof(T) + 128;
    static_assert((TXP * sizeof(T)) % 16 == 0, "TMA box inner extent must be a multiple of 16 B");
    static_assert(NSLOT >= 7, "ring must hold planes z-3..z+3");
};

template <typename T, int TX, int BY, int RY, int NSLOT, int ZC>
__global__ void __launch_bounds__(TX *BY)
diffusion_kernel(const __grid_constant__ CUtensorMap map_in, T *__restrict__ out, Geom g,
                 DC<T> c, int images, unsigned *err) {
    using Cfg = DiffCfg<T, TX, BY, RY, NSLOT, ZC>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations are kept 128-byte aligned (dynamic smem has 128 spare bytes)
    T *ring = reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    __shared__ __align__(8) uint64_t full[NSLOT];

    const int tx = threadIdx.x % TX, by = threadIdx.x / TX;
    const int64_t x0 = (int64_t)blockIdx.x * TX, y0 = (int64_t)blockIdx.y * Cfg::TY;
    const int64_t zc0 = (int64_t)blockIdx.z * ZC;
    const int64_t zend = min((int64_t)g.n[2], zc0 + ZC);
    const int nplanes = (int)(zend - zc0) + 2 * R6;  // planes zc0-3 .. zend+2
    const int64_t x = x0 + tx;
    const bool active_x = x < g.n[0];

    if (threadIdx.x == 0) {
        tma_prefetch_desc(&map_in);
        for (int s = 0; s < NSLOT; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    __syncthreads();

    // TMA box origin in padded coordinates: x start rounded down by HX (16-byte aligned),
    // y start = first halo row, z = padded plane index.
    const int bx = (int)(g.off[0] + x0 - Cfg::HX);
    const int by0 = (int)(g.off[1] + y0 - R6);
    const int bz0 = (int)(g.off[2] + zc0 - R6);
    auto issue = [&](int j) {  // load plane j (0-based from zc0-3) into slot j % NSLOT
        const int s = j % NSLOT;
        mbar_arrive_expect_tx(&full[s], Cfg::BOX_BYTES);
        tma_load_3d(ring + s * Cfg::SLOT_ELEMS, &map_in, &full[s], bx, by0, bz0 + j);
    };
    int issued = 0;
    if (threadIdx.x == 0)
        for (; issued < NSLOT && issued < nplanes; ++issued) issue(issued);

    T q[RY][7];
    bool ok = true;
    // centre of row r of this thread within a slot
    auto cell = [&](int slot, int r) -> T * {
        return ring + slot * Cfg::SLOT_ELEMS + (by * RY + r + R6) * Cfg::TXP + tx + Cfg::HX;
    };
    // prologue: own values of planes zc0-3 .. zc0+2 (j = 0..5)
    for (int j = 0; j < 2 * R6; ++j) {
        ok = ok && mbar_wait_bounded(&full[j % NSLOT], (j / NSLOT) & 1);
#pragma unroll
        for (int r = 0; r < RY; ++r) q[r][j + 1] = ok ? *cell(j % NSLOT, r) : T(0);
    }
    bool bad = __syncthreads_or(!ok);
    // planes j = 0..2 are no longer needed: refill their slots
    if (!bad && threadIdx.x == 0)
        for (; issued < NSLOT + R6 && issued < nplanes; ++issued) issue(issued);

    for (int m = 0; !bad && m < (int)(zend - zc0); ++m) {
        const int jl = m + 2 * R6;  // leading plane z+3
        const int sl = jl % NSLOT, sc = (m + R6) % NSLOT;
        ok = mbar_wait_bounded(&full[sl], (jl / NSLOT) & 1);
        if (ok) {
            const int64_t z = zc0 + m;
#pragma unroll
            for (int r = 0; r < RY; ++r) {
#pragma unroll
                for (int k = 0; k < 6; ++k) q[r][k] = q[r][k + 1];
                q[r][6] = *cell(sl, r);
                const T *p = cell(sc, r);
                T acc = c.g0 * q[r][3];
#pragma unroll
                for (int a = 1; a <= R6; ++a) {
                    acc = fma(c.ga[0][a - 1], p[a] + p[-a], acc);
                    acc = fma(c.ga[1][a - 1], p[a * Cfg::TXP] + p[-a * Cfg::TXP], acc);
                    acc = fma(c.ga[2][a - 1], q[r][3 + a] + q[r][3 - a], acc);
                }
                const int64_t y = y0 + by * RY + r;
                if (active_x && y < g.n[1]) store_with_images(out, g, R6, images != 0, x, y, z, acc);
            }
        }
        bad = __syncthreads_or(!ok);
        // plane j = m + 3 (centre of this iteration) is retired: reuse its slot
        if (!bad && threadIdx.x == 0 && issued < nplanes && issued == m + R6 + NSLOT) issue(issued++);
    }
    if (bad && threadIdx.x == 0) {
        atomicOr(err, ERR_TIMEOUT);
        // drain loads still in flight before the CTA's shared memory is released
        for (int j = max(0, issued - NSLOT); j < issued; ++j)
            (void)mbar_wait_bounded(&full[j % NSLOT], (j / NSLOT) & 1, 100000000ull);
    }
}

// ------------------------------------------------------------------ variants / launch

template <typename T, int TX, int BY, int RY, int NSLOT, int ZC>
static cudaError_t run(const CUtensorMap *map, void *out, const Geom &g, const DiffCoef &dc,
                       bool images, unsigned *err, cudaStream_t s) {
    using Cfg = DiffCfg<T, TX, BY, RY, NSLOT, ZC>;
    DC<T> c;
    c.g0 = (T)dc.g0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) c.ga[a][b] = (T)dc.ga[a][b];
    auto k = diffusion_kernel<T, TX, BY, RY, NSLOT, ZC>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((g.n[0] + TX - 1) / TX), (unsigned)((g.n[1] + Cfg::TY - 1) / Cfg::TY),
              (unsigned)((g.n[2] + ZC - 1) / ZC));
    k<<<grid, TX * BY, Cfg::SMEM, s>>>(*map, static_cast<T *>(out), g, c, images ? 1 : 0, err);
    return cudaGetLastError();
}

// Variant table: (TX, BY, RY, NSLOT, ZC) per dtype.  The autotuner times each on the
// problem and keeps the fastest.
#define DIFF_VARIANTS_F64(X) \
    X(32, 8, 1, 7, 64)       \
    X(32, 4, 2, 7, 64)       \
    X(64, 4, 1, 7, 64)       \
    X(32, 8, 1, 8, 32)
#define DIFF_VARIANTS_F32(X) \
    X(32, 8, 1, 8, 64)       \
    X(32, 4, 2, 8, 64)       \
    X(64, 4, 2, 8, 64)       \
    X(128, 2, 2, 9, 64)

int diffusion_num_variants(int dtype) { return dtype == 1 ? 4 : 4; }

const char *diffusion_variant_name(int dtype, int v) {
    static const char *f64[] = {"tx32_by8_ry1_s7_zc64", "tx32_by4_ry2_s7_zc64", "tx64_by4_ry1_s7_zc64",
                                "tx32_by8_ry1_s8_zc32"};
    static const char *f32[] = {"tx32_by8_ry1_s8_zc64", "tx32_by4_ry2_s8_zc64", "tx64_by4_ry2_s8_zc64",
                                "tx128_by2_ry2_s9_zc64"};
    if (v < 0 || v >= 4) return "?";
    return dtype == 1 ? f64[v] : f32[v];
}

void diffusion_box(int dtype, int v, int box[3]) {
    int i = 0;
    auto put = [&](int tx, int ty, int hx) {
        if (i++ == v) { box[0] = tx + 2 * hx; box[1] = ty + 2 * R6; box[2] = 1; }
    };
#define X(TX, BY, RY, NS, ZC) put(TX, BY * RY, 4);
    if (dtype == 1) { DIFF_VARIANTS_F64(X) } else { DIFF_VARIANTS_F32(X) }
#undef X
}

cudaError_t launch_diffusion(int dtype, const CUtensorMap *map, void *out, const Geom &g,
                             const DiffCoef &c, bool images, unsigned *err, cudaStream_t s,
                             int variant) {
    int i = 0;
    cudaError_t res = cudaErrorInvalidValue;
#define X(TX, BY, RY, NS, ZC) \
    if (i++ == variant) res = run<T, TX, BY, RY, NS, ZC>(map, out, g, c, images, err, s);
    if (dtype == 1) {
        using T = double;
        DIFF_VARIANTS_F64(X)
    } else if (dtype == 2) {
        using T = float;
        DIFF_VARIANTS_F32(X)
    }
#undef X
    return res;
}

}  // namespace stn
