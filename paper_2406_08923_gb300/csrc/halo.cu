// halo.cu -- periodic halo fill of augmented arrays (Sec. 2.4, Eq. 2 with periodic beta).
//
// One launch fills every halo cell of up to 8 fields directly from the interior cell it
// images (index arithmetic modulo the interior extent on each axis), so no ordering between
// faces, edges and corners is needed.  Grid: x = blocks striding over the halo cells of one
// padded z-plane, y = padded z-plane, z = field.
//
// With zwrap = 0 (x and y periodic, the z halo supplied by the caller, as in a z-slab of a
// decomposed grid) every padded plane, the z-halo planes included, gets the x/y periodic
// images of its own cells and no plane is copied along z.
#include "internal.h"

namespace stn {

template <typename T>
__global__ void halo_fill_kernel(Ptrs8 f, Geom g, int r, int zwrap) {
    T *base = static_cast<T *>(f.p[blockIdx.z]);
    const int64_t nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int64_t hy = ny > 1 ? r : 0, hz = nz > 1 ? r : 0;
    const int64_t wx = nx + 2 * r, wy = ny + 2 * hy;
    const int64_t kr = blockIdx.y;  // z in the used range [0, nz + 2 hz)
    const bool halo_plane = zwrap && ((kr < hz) || (kr >= nz + hz));
    const int64_t count = halo_plane ? wx * wy : 2 * hy * wx + ny * 2 * r;
    const int64_t sk = zwrap ? ((kr - hz) % nz + nz) % nz : kr - hz;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t xr, yr;
        if (halo_plane) {
            yr = q / wx;
            xr = q - yr * wx;
        } else if (q < 2 * hy * wx) {
            int64_t row = q / wx;
            xr = q - row * wx;
            yr = row < hy ? row : ny + row;  // rows [0, hy) and [ny + hy, ny + 2 hy)
        } else {
            int64_t q2 = q - 2 * hy * wx;
            int64_t row = q2 / (2 * r), c = q2 - row * (2 * r);
            yr = hy + row;
            xr = c < r ? c : nx + c;  // columns [0, r) and [nx + r, nx + 2 r)
        }
        const int64_t sx = ((xr - r) % nx + nx) % nx;
        const int64_t sy = ((yr - hy) % ny + ny) % ny;
        const int64_t dst = (g.off[0] - r + xr) + g.pad[0] * ((g.off[1] - hy + yr) +
                                                               g.pad[1] * (g.off[2] - hz + kr));
        base[dst] = base[g.idx(sx, sy, sk)];
    }
}

cudaError_t launch_halo_fill(const Geom &g, int r, int esize, const Ptrs8 &f, int nfields,
                             cudaStream_t s, bool zwrap) {
    if (r == 0) return cudaSuccess;
    const int64_t hz = g.n[2] > 1 ? r : 0;
    dim3 grid(1, (unsigned)(g.n[2] + 2 * hz), (unsigned)nfields);
    const int64_t per_plane = (g.n[0] + 2 * r) * (g.n[1] + 2 * (g.n[1] > 1 ? r : 0));
    grid.x = (unsigned)std::min<int64_t>(64, (per_plane + 255) / 256);
    switch (esize) {
    case 2: halo_fill_kernel<uint16_t><<<grid, 256, 0, s>>>(f, g, r, zwrap ? 1 : 0); break;
    case 4: halo_fill_kernel<uint32_t><<<grid, 256, 0, s>>>(f, g, r, zwrap ? 1 : 0); break;
    case 8: halo_fill_kernel<uint64_t><<<grid, 256, 0, s>>>(f, g, r, zwrap ? 1 : 0); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Failure-detection self-test: wait on an mbarrier that never completes (nothing arrives and
// no transaction bytes are expected), bounded by limit_ns, and report the expiry.
__global__ void selftest_wait_kernel(uint64_t limit_ns, unsigned *err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
}

cudaError_t launch_selftest_wait(uint64_t limit_ns, unsigned *err, cudaStream_t s) {
    selftest_wait_kernel<<<1, 32, 0, s>>>(limit_ns, err);
    return cudaGetLastError();
}

}  // namespace stn
