// internal.h -- declarations shared between the C-ABI layer (api.cu) and the kernel files.
#pragma once

#include "common.cuh"
#include "persist.cuh"

namespace stn {

// Launch `k` with programmatic stream serialization (see pdl_wait in common.cuh): the kernel
// must call pdl_wait() before its first global-memory access.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, static_cast<Args &&>(args)...);
}

struct Ptrs8 {
    void *p[8];
};

// Periodic halo fill (Eq. 2, periodic beta) of `nfields` fields of element size `esize`.
// zwrap = false: x/y images only, on every padded plane (z halo owned by the caller).
cudaError_t launch_halo_fill(const Geom &g, int r, int esize, const Ptrs8 &f, int nfields,
                             cudaStream_t s, bool zwrap = true);

// XCORR (Eq. 3): `sweeps` sweeps in one launch.  dtype: 0 = int32 (mod 2^32), 1 = f64,
// 2 = f32.  periodic: halo read by wrapping interior indices (any sweeps <= max);
// otherwise a single sweep reading the caller's halo.  images: write periodic images of
// the output into its halo.
int xcorr_max_sweeps_per_launch(int r);
cudaError_t launch_xcorr(int dtype, int r, const void *in, void *out, const Geom &g,
                         const void *coeffs, int sweeps, bool periodic, bool images,
                         cudaStream_t s);

// XCORR of radius 5..1024 (register-blocked, weights in device memory `wdev`, dtype 1 = f64,
// 2 = f32) and the max filter (radius 0..1024, dtype 0 = int32, 1 = f64, 2 = f32); one sweep
// per launch (xcorr_wide.cu).
int xcorr_wide_max_radius();
cudaError_t launch_xcorr_wide(int dtype, int r, const void *in, void *out, const Geom &g, const void *wdev,
                              bool periodic, bool images, unsigned *err, cudaStream_t s);
cudaError_t launch_maxfilter(int dtype, int r, const void *in, void *out, const Geom &g, bool periodic, bool images,
                             unsigned *err, cudaStream_t s);

// Grid sizing shared by the z-streaming kernels: number of z-chunks that best fills whole
// waves of `slots` resident CTAs (see diffusion.cu), and the SM count of the current device.
int choose_zchunks(int tiles, int nz, int slots, double reread_weight);
// z-chunk length of a launch: the kernel's own choice `zc` (zmode 0), half of it (zmode 1, more
// and shorter chunks) or twice it (zmode 2, fewer and longer), within 1..nz.  The autotuner
// searches the mode next to the tile shape.
int zchunk_len(int zc, int nz, int zmode);
constexpr int ZMODES = 3;
int device_sms();

// DIFFUSION (Eqs. 4-7): one folded forward-Euler step with the order-2r central Laplacian of
// radius r = 1..4 (r = 3: the 6th-order, 19-point stencil in 3D).  1D runs through the XCORR
// kernel with the folded weights; 2D and 3D have their own kernels, reading through TMA.
struct DiffCoef {
    double g0;        // centre weight 1 + dt*alpha*sum_axes c0/h^2
    double ga[3][4];  // [axis][a-1] weight of the pair at offset +-a along axis (0 beyond r)
    int r;            // radius 1..4
};
// 3D
cudaError_t launch_diffusion(int dtype, const CUtensorMap *map_in, void *out, const Geom &g,
                             const DiffCoef &c, bool images, unsigned *err, cudaStream_t s,
                             int variant, int zmode = 0);
int diffusion_num_variants(int dtype, int r);
const char *diffusion_variant_name(int dtype, int r, int variant);
void diffusion_box(int dtype, int r, int variant, int box[3]);  // TMA box (x, y, z) of a variant
// Persistent variants run all nsteps steps of a call in one cooperative launch (persist.cuh):
// step s reads the field written by step s-1 (maps[0], the input, for s = 0) and writes `out`
// when nsteps - 1 - s is even, `tmp` otherwise; maps = {in, tmp, out}.  `sync` is a zeroed
// buffer of at least PERSIST_HDR + units 64-bit words kept between calls; with sync == nullptr
// the call only reports the launch's unit count in *units.
bool diffusion_persistent(int dtype, int r, int variant);
cudaError_t launch_diffusion_persist(int dtype, const CUtensorMap *maps, void *tmp, void *out, const Geom &g,
                                     const DiffCoef &c, bool images, int nsteps, unsigned long long *sync,
                                     int64_t sync_words, unsigned *err, cudaStream_t s, int variant, int zmode,
                                     int64_t *units);
// The FP32 kernel family (diffusion_f32.cu), reached through the functions above for dtype 2.
int diffusion_f32_num_variants(int r);
const char *diffusion_f32_variant_name(int r, int variant);
void diffusion_f32_box(int r, int variant, int box[3]);
cudaError_t launch_diffusion_f32(const CUtensorMap *map_in, float *out, const Geom &g, const DiffCoef &c,
                                 bool images, unsigned *err, cudaStream_t s, int variant, int zmode = 0);
bool diffusion_f32_persistent(int r, int variant);
cudaError_t launch_diffusion_f32_persist(const CUtensorMap *maps, float *tmp, float *out, const Geom &g,
                                         const DiffCoef &c, bool images, int nsteps, unsigned long long *sync,
                                         int64_t sync_words, unsigned *err, cudaStream_t s, int variant, int zmode,
                                         int64_t *units);
// 2D (diffusion2d.cu): one TMA tile per CTA, no streaming axis.
cudaError_t launch_diffusion2d(int dtype, const CUtensorMap *map_in, void *out, const Geom &g, const DiffCoef &c,
                               bool images, unsigned *err, cudaStream_t s);
void diffusion2d_box(int dtype, int r, int box[3]);
// 2D, temporally blocked (diffusion2d_tb.cu): `steps` = 2 or 4 Euler steps per pass, FP32,
// periodic, nx a multiple of 4 (diffusion2d_tb_ok); reads `in` with periodic wrap (no halo).
bool diffusion2d_tb_ok(int dtype, const Geom &g);
cudaError_t launch_diffusion2d_tb(int dtype, int steps, const void *in, void *out, const Geom &g, const DiffCoef &c,
                                  cudaStream_t s);

// MHD8 (Eqs. A1-A4 + RK3).  Constants in the compute type are built inside mhd.cu.
struct MhdConst {
    double d1[3][3], d2c[3], d2[3][3], dm[3][3];  // scaled stencil weights
    double cs0sq, gamma, inv_cp, lnrho0, nu, eta, zeta, mu0, inv_mu0, cp_gm1;
    double K;  // heat conductivity of Eq. A3 (0: no conduction term)
    double dt;
};
struct MhdMaps {
    CUtensorMap m[8];
};

// mode 0: RK substep `sub` (0..2) writing f_out (+images), w and (for Kahan) c;
// mode 1: right-hand side only, written densely to rhs (compute type).
// The RK register w and the Kahan terms c are one array each, in the storage type, with the 8
// fields of a cell next to each other (element 8 cell + q; `cell` the dense interior index),
// so a cell's 8 values move as 16-byte vectors.
cudaError_t launch_mhd(int storage, int mode, int sub, const MhdMaps &maps, const Ptrs8 &fout,
                       void *w, void *kc, const Ptrs8 &rhs, const Geom &g,
                       const MhdConst &k, bool images, unsigned *err, cudaStream_t s,
                       int variant, int zmode = 0);
void mhd_box(int storage, int variant, int box[3]);
int mhd_num_variants(int storage);
const char *mhd_variant_name(int storage, int variant);

// Norms: two-pass deterministic FP64 reduction.  partials holds nblocks * nfields * 4.
int norms_blocks();
cudaError_t launch_norms(int storage, const Ptrs8 &f, int nfields, const Geom &g, bool mass0,
                         double *partials, double *out_dev, cudaStream_t s);

// Bounded-wait self-test: one CTA waits on an mbarrier nothing completes.
cudaError_t launch_selftest_wait(uint64_t limit_ns, unsigned *err, cudaStream_t s);

// Allocation-free norms: partials in a file-scope device array (norms.cu); results packed
// {sum, sumsq, max|f|} per field (+ mass) into device memory.
int norms_static_max_fields();
cudaError_t launch_norms_noalloc(int storage, const Ptrs8 &f, int nfields, const Geom &g,
                                 double mass_volume, double *out_dev, cudaStream_t s);

// ------------------------------------------------------------------ batched serving
// Scaled MHD constants in the compute type (defined here so batched work items can carry
// them); alpha/beta are the RK substep coefficients.
template <typename C> struct MK {
    C d1[3][3], d2c[3], d2[3][3], dm[3][3];
    C cs0sq, gamma, inv_cp, lnrho0, nu, eta, zeta, mu0, inv_mu0, cp_gm1;
    C K;
    C dt, alpha, beta;
    // derived constants, so that every operand of the explicit arithmetic is a member
    C gcp, gm1, etamu0, two_nu;  // gamma / cp, gamma - 1, eta mu0, 2 nu
    C one, mone, half, two, third, mthird;
};

// Work items of one batched launch.  Every item owns a contiguous range of virtual CTAs
// [cta_begin, cta_begin + tiles); a persistent grid strides over the virtual CTAs and finds
// the item by binary search on cta_begin.  All pointers are device pointers; descriptors are
// resident in device memory (64-byte aligned).  Storage and arithmetic are FP32.
struct BatchHeat {
    const CUtensorMap *map;  // source field
    float *out;
    Geom g;
    float g0, ga[3][3];
    int zc, tiles_x, tiles_y, tiles_z;
    int cta_begin, pad_;
};
struct BatchMhd {
    const CUtensorMap *maps;  // 8 consecutive descriptors of the source field set
    Ptrs8 fout;
    float *w, *kc;  // RK register and Kahan terms, 8 fields interleaved per cell (launch_mhd)
    Geom g;
    MK<float> k;  // alpha/beta filled in per launch
    int zc, tiles_x, tiles_y, tiles_z;
    int cta_begin, pad_;
};
struct BatchXcorr {
    const float *in;
    float *out;
    Geom g;
    float w[7];  // weights g_{-3..3}
    int chunks;
    int cta_begin, pad_;
};
// Counts of one batched iteration (device memory, read by the persistent kernels).
struct BatchHeader {
    int n_heat, heat_ctas, n_mhd, mhd_ctas, n_xc, xc_ctas, pad_[2];
};

// `shape`: the batched kernel's tile shape, 0 or 1 (see diffusion_f32.cu / mhd.cu)
cudaError_t launch_diffusion_batch(int shape, const BatchHeader *hdr, const BatchHeat *items, unsigned *err, int grid,
                                   cudaStream_t s);
cudaError_t launch_mhd_batch(int shape, const BatchHeader *hdr, const BatchMhd *items, int sub, unsigned *err,
                             int grid, cudaStream_t s);
cudaError_t launch_xcorr_batch(const BatchHeader *hdr, const BatchXcorr *items, unsigned *err, int grid,
                               cudaStream_t s);
// persistent grid sizes (resident CTAs on the current device) and tile shapes of the batched kernels
int diffusion_batch_grid(int shape);
int mhd_batch_grid(int shape);
int xcorr_batch_grid();
void diffusion_batch_tile(int shape, int *tx, int *ty, int box[3]);
void mhd_batch_tile(int shape, int *tx, int *ty, int box[3]);
const char *diffusion_batch_shape_name(int shape);
const char *mhd_batch_shape_name(int shape);
// The batched tile shape (0 or 1) matching the tile of the per-grid variant the autotuner
// last chose for FP32 plans of `kind` (STENCIL_DIFFUSION or STENCIL_MHD8) on the current
// device, in this process or in the autotuning cache file; -1 if nothing was tuned (api.cu).
int tuned_batch_shape(int kind);
int xcorr_batch_chunk();
void mhd_scaled_constants(const MhdConst &c, MK<float> *k);
// FP32 constants of RK substep `sub` (its alpha and beta filled in)
void mhd_substep_constants(const MhdConst &c, int sub, MK<float> *k);

}  // namespace stn
