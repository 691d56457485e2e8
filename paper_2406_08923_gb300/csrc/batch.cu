// batch.cu -- continuous-batching server: many independent stencil problems of different
// kinds and sizes resident on the device at once, advanced together by batched persistent
// kernels (one launch per kind and step for all active problems).
//
// Scheduling model (one call of stencil_server_progress = one iteration):
//   1. retire: problems whose result copy-back event has completed are marked done and their
//      device memory is returned to the stream-ordered pool;
//   2. admit: pending problems, in arrival order, are admitted while the HBM byte budget and
//      the active-slot limit allow; admission allocates one pool block per problem (fields,
//      RK register, Kahan terms, TMA descriptors), uploads the initial fields and packs them
//      into the padded periodic layout (Eq. 2) on the device;
//   3. step: every active problem advances one step -- one heat Euler step, one RK3 step of
//      the MHD system (three substep launches) or one cross-correlation sweep -- through a
//      work table uploaded from pinned memory and one persistent batched launch per kind;
//   4. finish: problems that reached their step count are unpacked on the device and copied
//      back to the caller's host arrays; an event marks completion.
// Problems admitted in iteration i start stepping in iteration i, so requests that arrive
// while others run join the batch as slots and memory free up.  All storage and arithmetic
// is FP32 (the serving configuration), with Kahan-compensated RK for MHD.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/stencil.h"
#include "internal.h"

using namespace stn;

namespace {

constexpr int R = 3;

// dense (nz, ny, nx) FP32 -> padded periodic layout, halo included
__global__ void pack_periodic_kernel(const float *__restrict__ dense, float *__restrict__ padded, Geom g) {
    const int64_t hx = R, hy = g.n[1] > 1 ? R : 0, hz = g.n[2] > 1 ? R : 0;
    const int64_t wx = g.n[0] + 2 * hx, wy = g.n[1] + 2 * hy, wz = g.n[2] + 2 * hz;
    const int64_t total = wx * wy * wz;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t xr = q % wx, t = q / wx, yr = t % wy, zr = t / wy;
        const int64_t sx = ((xr - hx) % g.n[0] + g.n[0]) % g.n[0];
        const int64_t sy = ((yr - hy) % g.n[1] + g.n[1]) % g.n[1];
        const int64_t sz = ((zr - hz) % g.n[2] + g.n[2]) % g.n[2];
        padded[(g.off[0] - hx + xr) + g.pad[0] * ((g.off[1] - hy + yr) + g.pad[1] * (g.off[2] - hz + zr))] =
            dense[sx + g.n[0] * (sy + g.n[1] * sz)];
    }
}

// padded interior -> dense (nz, ny, nx)
__global__ void unpack_kernel(const float *__restrict__ padded, float *__restrict__ dense, Geom g) {
    const int64_t total = g.n[0] * g.n[1] * g.n[2];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = q % g.n[0], t = q / g.n[0], y = t % g.n[1], z = t / g.n[1];
        dense[q] = padded[g.idx(x, y, z)];
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool encode_f32(CUtensorMap *m, const float *ptr, const Geom &g, const int box[3]) {
    auto fn = encoder();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)g.pad[0], (cuuint64_t)g.pad[1], (cuuint64_t)g.pad[2]};
    cuuint64_t strides[2] = {(cuuint64_t)(g.pad[0] * 4), (cuuint64_t)(g.pad[0] * g.pad[1] * 4)};
    cuuint32_t bx[3] = {(cuuint32_t)box[0], (cuuint32_t)box[1], (cuuint32_t)box[2]};
    cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(ptr), dims, strides, bx, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

enum { ST_PENDING = 0, ST_ACTIVE = 1, ST_COMPLETING = 2, ST_DONE = 3, ST_CANCELLED = 4 };

struct Req {
    int64_t ticket = 0;
    stencil_kind kind = STENCIL_DIFFUSION;
    int state = ST_PENDING;
    int nsteps = 0, steps_done = 0, nf = 1, cur = 0;
    Geom g{};
    int64_t ncell = 0, field_elems = 0;
    size_t bytes = 0;
    void *base = nullptr;
    float *set[2][8] = {};
    float *w = nullptr, *kc = nullptr;  // RK register and Kahan terms, 8 fields interleaved per cell
    CUtensorMap *dmaps = nullptr;  // [2][nf] descriptors in device memory
    CUtensorMap hmaps[16];         // host copy the upload reads from (lives as long as the request)
    int tiles[3] = {1, 1, 1}, zc = 1;
    float g0 = 0, ga[3][3] = {};
    MK<float> k{};
    float w7[7] = {};
    const float *host_in[8] = {};
    float *host_out[8] = {};
    cudaEvent_t ev = nullptr;
};

}  // namespace

struct stencil_server {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaMemPool_t pool = nullptr;
    int64_t budget = 0, used = 0, peak = 0;
    int max_active = 0;
    int64_t next_ticket = 1;
    int64_t cell_updates = 0;  // cells x steps of all finished problems
    std::deque<Req *> pending;
    std::vector<Req *> active;      // ST_ACTIVE
    std::vector<Req *> completing;  // ST_COMPLETING
    std::unordered_map<int64_t, Req *> table;
    // work tables: pinned host (double-buffered) and device
    size_t table_bytes = 0;
    unsigned char *host_tab[2] = {};
    cudaEvent_t tab_ev[2] = {};
    int tab_i = 0;
    unsigned char *dev_tab = nullptr;
    unsigned *err = nullptr;
    int grid_heat = 0, grid_mhd = 0, grid_xc = 0;
    int heat_shape = 0, mhd_shape = 0;  // tile shapes of the batched heat / MHD kernels
    bool own_stream = false;
    // one captured graph per pinned table buffer: table upload + every batched launch
    cudaGraph_t graph[2] = {};  // kept alive: exec node updates refer to its nodes
    cudaGraphExec_t exec[2] = {};
    cudaGraphNode_t copy_node[2] = {};
    std::string detail;
};

namespace {

thread_local std::string g_server_detail;

stencil_status sfail(stencil_server_t s, stencil_status st, const std::string &m) {
    if (s) s->detail = m;
    else g_server_detail = m;
    return st;
}

stencil_status scuda(stencil_server_t s, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    cudaGetLastError();
    return sfail(s, e == cudaErrorMemoryAllocation ? STENCIL_ENOMEM : STENCIL_ECUDA, m);
}

#define SCK(s, call, what)                                  \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return scuda(s, e_, what);   \
    } while (0)

// layout of one FP32 field of a problem (same rule as stencil_layout)
Geom layout_f32(int ndim, const int64_t dims[3]) {
    Geom g{};
    const int64_t xoff = 4, align = 8;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = a < ndim ? dims[a] : 1;
        g.off[a] = a == 0 ? xoff : (a < ndim ? R : 0);
    }
    g.pad[0] = ((xoff + g.n[0] + xoff + align - 1) / align) * align;
    g.pad[1] = ndim >= 2 ? g.n[1] + 2 * R : 1;
    g.pad[2] = ndim >= 3 ? g.n[2] + 2 * R : 1;
    return g;
}

size_t table_size(int max_active) {
    return up256(sizeof(BatchHeader)) + up256(sizeof(BatchHeat) * max_active) +
           3 * up256(sizeof(BatchMhd) * max_active) + up256(sizeof(BatchXcorr) * max_active);
}

stencil_status admit(stencil_server_t s, Req *r) {
    cudaStream_t st = s->stream;
    SCK(s, cudaMallocFromPoolAsync(&r->base, r->bytes, s->pool, st), "pool allocation");
    // carve the block: fields (2 sets), RK register and Kahan terms, descriptors
    unsigned char *p = static_cast<unsigned char *>(r->base);
    const size_t fb = up256(r->field_elems * sizeof(float));
    for (int k = 0; k < 2; ++k)
        for (int q = 0; q < r->nf; ++q, p += fb) r->set[k][q] = reinterpret_cast<float *>(p);
    if (r->kind == STENCIL_MHD8) {
        const size_t db = up256(r->ncell * sizeof(float));
        r->w = reinterpret_cast<float *>(p);
        p += 8 * db;
        r->kc = reinterpret_cast<float *>(p);
        p += 8 * db;
    }
    r->dmaps = reinterpret_cast<CUtensorMap *>(p);
    // upload the dense initial fields into set 1 (as staging), pack into set 0 with halos
    for (int q = 0; q < r->nf; ++q) {
        SCK(s, cudaMemcpyAsync(r->set[1][q], r->host_in[q], r->ncell * sizeof(float), cudaMemcpyHostToDevice, st),
            "upload");
        const int blocks = (int)std::min<int64_t>(1024, (r->field_elems + 255) / 256);
        pack_periodic_kernel<<<blocks, 256, 0, st>>>(r->set[1][q], r->set[0][q], r->g);
        SCK(s, cudaGetLastError(), "pack launch");
    }
    if (r->kind == STENCIL_MHD8)
        SCK(s, cudaMemsetAsync(r->kc, 0, 8 * r->ncell * sizeof(float), st), "clear Kahan");
    // TMA descriptors of both field sets
    if (r->kind != STENCIL_XCORR) {
        int box[3], tx, ty;
        if (r->kind == STENCIL_DIFFUSION) diffusion_batch_tile(s->heat_shape, &tx, &ty, box);
        else mhd_batch_tile(s->mhd_shape, &tx, &ty, box);
        for (int k = 0; k < 2; ++k)
            for (int q = 0; q < r->nf; ++q)
                if (!encode_f32(&r->hmaps[k * r->nf + q], r->set[k][q], r->g, box))
                    return sfail(s, STENCIL_ECUDA, "cuTensorMapEncodeTiled failed");
        SCK(s, cudaMemcpyAsync(r->dmaps, r->hmaps, sizeof(CUtensorMap) * 2 * r->nf, cudaMemcpyHostToDevice, st),
            "descriptor upload");
    }
    r->cur = 0;
    r->state = ST_ACTIVE;
    s->used += (int64_t)r->bytes;
    s->peak = std::max(s->peak, s->used);
    s->active.push_back(r);
    return STENCIL_OK;
}

stencil_status finish(stencil_server_t s, Req *r) {
    cudaStream_t st = s->stream;
    const int other = r->cur ^ 1;
    for (int q = 0; q < r->nf; ++q) {
        const int blocks = (int)std::min<int64_t>(1024, (r->ncell + 255) / 256);
        unpack_kernel<<<blocks, 256, 0, st>>>(r->set[r->cur][q], r->set[other][q], r->g);
        SCK(s, cudaGetLastError(), "unpack launch");
        SCK(s, cudaMemcpyAsync(r->host_out[q], r->set[other][q], r->ncell * sizeof(float), cudaMemcpyDeviceToHost,
                               st),
            "download");
    }
    SCK(s, cudaEventRecord(r->ev, st), "completion event");
    r->state = ST_COMPLETING;
    s->completing.push_back(r);
    return STENCIL_OK;
}

struct TableLayout {
    size_t off_heat, off_mhd, mhd_stride, off_xc;
};

TableLayout table_layout(int max_active) {
    TableLayout t;
    t.off_heat = up256(sizeof(BatchHeader));
    t.off_mhd = t.off_heat + up256(sizeof(BatchHeat) * max_active);
    t.mhd_stride = up256(sizeof(BatchMhd) * max_active);
    t.off_xc = t.off_mhd + 3 * t.mhd_stride;
    return t;
}

// Capture, for each pinned table buffer, one iteration: table upload followed by the
// persistent batched launches of every kind.  The grids are occupancy-sized and the kernels
// read their work counts from the uploaded table, so one graph serves every batch; only the
// upload size changes between replays.
stencil_status capture_graphs(stencil_server_t s) {
    const TableLayout t = table_layout(s->max_active);
    const BatchHeader *dhdr = reinterpret_cast<const BatchHeader *>(s->dev_tab);
    for (int i = 0; i < 2; ++i) {
        cudaGraph_t graph = nullptr;
        SCK(s, cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t e = cudaMemcpyAsync(s->dev_tab, s->host_tab[i], s->table_bytes, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess)
            e = launch_diffusion_batch(s->heat_shape, dhdr, reinterpret_cast<const BatchHeat *>(s->dev_tab + t.off_heat),
                                       s->err, s->grid_heat, s->stream);
        for (int sub = 0; sub < 3 && e == cudaSuccess; ++sub)
            e = launch_mhd_batch(s->mhd_shape, dhdr,
                                 reinterpret_cast<const BatchMhd *>(s->dev_tab + t.off_mhd + sub * t.mhd_stride), sub,
                                 s->err, s->grid_mhd, s->stream);
        if (e == cudaSuccess)
            e = launch_xcorr_batch(dhdr, reinterpret_cast<const BatchXcorr *>(s->dev_tab + t.off_xc), s->err,
                                   s->grid_xc, s->stream);
        cudaError_t e2 = cudaStreamEndCapture(s->stream, &graph);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return scuda(s, e, "capture of the batched iteration");
        }
        SCK(s, e2, "end capture");
        // find the memcpy node (the graph's only root)
        size_t nroot = 0;
        e = cudaGraphGetRootNodes(graph, nullptr, &nroot);
        cudaGraphNode_t root = nullptr;
        if (e == cudaSuccess && nroot == 1) e = cudaGraphGetRootNodes(graph, &root, &nroot);
        if (e == cudaSuccess && nroot != 1) e = cudaErrorInvalidValue;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&s->exec[i], graph, 0);
        s->graph[i] = graph;
        SCK(s, e, "graph instantiation");
        s->copy_node[i] = root;
    }
    return STENCIL_OK;
}

}  // namespace

extern "C" {

stencil_status stencil_server_create(int64_t hbm_budget_bytes, int max_active, void *stream, stencil_server_t *out) {
    g_server_detail.clear();
    if (!out) return sfail(nullptr, STENCIL_EINVAL, "out is NULL");
    *out = nullptr;
    if (hbm_budget_bytes <= 0) return sfail(nullptr, STENCIL_EINVAL, "budget must be positive");
    if (max_active < 1 || max_active > 65536) return sfail(nullptr, STENCIL_EINVAL, "max_active out of range 1..65536");
    stencil_server *s = new (std::nothrow) stencil_server;
    if (!s) return sfail(nullptr, STENCIL_ENOMEM, "host allocation failed");
    s->budget = hbm_budget_bytes;
    s->max_active = max_active;
    s->stream = (cudaStream_t)stream;
    if (!s->stream) {  // graphs cannot be captured on the legacy default stream
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return sfail(nullptr, STENCIL_ECUDA, "cudaStreamCreate failed");
        }
        s->own_stream = true;
    }
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetDefaultMemPool(&s->pool, s->device);
    if (e == cudaSuccess) {
        uint64_t thr = UINT64_MAX;  // keep freed blocks in the pool for reuse
        e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    s->table_bytes = table_size(max_active);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaMallocHost((void **)&s->host_tab[i], s->table_bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->tab_ev[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->dev_tab, s->table_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(s->err, 0, sizeof(unsigned));
    if (e != cudaSuccess) {
        stencil_status st = scuda(nullptr, e, "server set-up");
        stencil_server_destroy(s);
        return st;
    }
    // tile shapes: the autotuner's latest choice for FP32 plans of the kind on this GPU (the
    // batched kernels run the same tile code as the per-grid ones), else the default shape
    s->heat_shape = std::max(0, tuned_batch_shape(STENCIL_DIFFUSION));
    s->mhd_shape = std::max(0, tuned_batch_shape(STENCIL_MHD8));
    s->grid_heat = diffusion_batch_grid(s->heat_shape);
    s->grid_mhd = mhd_batch_grid(s->mhd_shape);
    s->grid_xc = xcorr_batch_grid();
    stencil_status gst = capture_graphs(s);
    if (gst != STENCIL_OK) {
        g_server_detail = s->detail;
        stencil_server_destroy(s);
        return gst;
    }
    *out = s;
    return STENCIL_OK;
}

void stencil_server_destroy(stencil_server_t s) {
    if (!s) return;
    if (s->stream || s->dev_tab) cudaStreamSynchronize(s->stream);
    for (auto &kv : s->table) {
        Req *r = kv.second;
        if (r->base) cudaFreeAsync(r->base, s->stream);
        if (r->ev) cudaEventDestroy(r->ev);
        delete r;
    }
    cudaStreamSynchronize(s->stream);
    for (int i = 0; i < 2; ++i) {
        if (s->host_tab[i]) cudaFreeHost(s->host_tab[i]);
        if (s->tab_ev[i]) cudaEventDestroy(s->tab_ev[i]);
    }
    for (int i = 0; i < 2; ++i) {
        if (s->exec[i]) cudaGraphExecDestroy(s->exec[i]);
        if (s->graph[i]) cudaGraphDestroy(s->graph[i]);
    }
    if (s->dev_tab) cudaFree(s->dev_tab);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    if (s->err) cudaFree(s->err);
    delete s;
}

stencil_status stencil_server_submit(stencil_server_t s, const stencil_request *req, const float *const *host_in,
                                     float *const *host_out, int64_t *ticket) {
    if (!s) return sfail(nullptr, STENCIL_EINVAL, "server is NULL");
    if (!req || !host_in || !host_out || !ticket) return sfail(s, STENCIL_EINVAL, "a pointer argument is NULL");
    Req *r = new (std::nothrow) Req;
    if (!r) return sfail(s, STENCIL_ENOMEM, "host allocation failed");
    r->kind = req->kind;
    r->nsteps = req->nsteps;
    int ndim;
    switch (req->kind) {
    case STENCIL_XCORR: ndim = 1; r->nf = 1; break;
    case STENCIL_DIFFUSION: ndim = 3; r->nf = 1; break;
    case STENCIL_MHD8: ndim = 3; r->nf = 8; break;
    default: delete r; return sfail(s, STENCIL_EINVAL, "unknown kind");
    }
    if (req->nsteps < 1) { delete r; return sfail(s, STENCIL_EINVAL, "nsteps must be >= 1"); }
    const int64_t dmax = ndim == 1 ? ((int64_t)1 << 31) - 16 : ((int64_t)1 << 15);
    for (int a = 0; a < ndim; ++a)
        if (req->dims[a] < 2 * R + 1 || req->dims[a] > dmax) {
            delete r;
            return sfail(s, STENCIL_EINVAL, ndim == 1 ? "1D extent must be in 7 .. 2^31-16 (periodic, radius 3)"
                                                      : "3D extents must be in 7 .. 2^15 (periodic, radius 3)");
        }
    for (int q = 0; q < r->nf; ++q)
        if (!host_in[q] || !host_out[q]) { delete r; return sfail(s, STENCIL_EINVAL, "host field pointer is NULL"); }
    r->g = layout_f32(ndim, req->dims);
    r->ncell = r->g.n[0] * r->g.n[1] * r->g.n[2];
    r->field_elems = r->g.pad[0] * r->g.pad[1] * r->g.pad[2];
    for (int q = 0; q < r->nf; ++q) {
        r->host_in[q] = host_in[q];
        r->host_out[q] = host_out[q];
    }
    // constants and tiling
    const stencil_params &p = req->params;
    if (req->kind == STENCIL_XCORR) {
        for (int j = 0; j < 7; ++j) r->w7[j] = (float)req->coeffs[j];
        r->tiles[0] = (int)((r->ncell + xcorr_batch_chunk() - 1) / xcorr_batch_chunk());
    } else {
        for (int a = 0; a < 3; ++a)
            if (!(p.dx[a] > 0.0)) { delete r; return sfail(s, STENCIL_EINVAL, "grid spacing must be positive"); }
        static const double W1[3] = {3.0 / 4.0, -3.0 / 20.0, 1.0 / 60.0};
        static const double W2C = -49.0 / 18.0;
        static const double W2[3] = {3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0};
        static const double WM[3] = {270.0, -27.0, 2.0};
        int tx, ty, box[3];
        if (req->kind == STENCIL_DIFFUSION) {
            const double sc = p.dt * p.alpha;
            double g0 = 1.0;
            for (int a = 0; a < 3; ++a) {
                g0 += sc * W2C / (p.dx[a] * p.dx[a]);
                for (int i = 0; i < 3; ++i) r->ga[a][i] = (float)(sc * W2[i] / (p.dx[a] * p.dx[a]));
            }
            r->g0 = (float)g0;
            diffusion_batch_tile(s->heat_shape, &tx, &ty, box);
        } else {
            if (!(p.cp > 0.0) || !(p.gamma > 1.0) || !(p.mu0 > 0.0)) {
                delete r;
                return sfail(s, STENCIL_EINVAL, "MHD8 needs cp > 0, gamma > 1, mu0 > 0");
            }
            MhdConst c{};
            const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
            for (int a = 0; a < 3; ++a) {
                c.d2c[a] = W2C / (p.dx[a] * p.dx[a]);
                for (int i = 0; i < 3; ++i) {
                    c.d1[a][i] = W1[i] / p.dx[a];
                    c.d2[a][i] = W2[i] / (p.dx[a] * p.dx[a]);
                    c.dm[a][i] = WM[i] / (720.0 * p.dx[pairs[a][0]] * p.dx[pairs[a][1]]);
                }
            }
            c.cs0sq = p.cs0 * p.cs0; c.gamma = p.gamma; c.inv_cp = 1.0 / p.cp; c.lnrho0 = p.lnrho0;
            c.nu = p.nu; c.eta = p.eta; c.zeta = p.zeta; c.mu0 = p.mu0; c.inv_mu0 = 1.0 / p.mu0;
            c.cp_gm1 = p.cp * (p.gamma - 1.0); c.K = p.K; c.dt = p.dt;
            mhd_scaled_constants(c, &r->k);
            mhd_batch_tile(s->mhd_shape, &tx, &ty, box);
        }
        const int nz = (int)r->g.n[2];
        r->zc = std::min(nz, 32);
        r->tiles[0] = (int)((r->g.n[0] + tx - 1) / tx);
        r->tiles[1] = (int)((r->g.n[1] + ty - 1) / ty);
        r->tiles[2] = (nz + r->zc - 1) / r->zc;
    }
    // device bytes held while resident
    size_t b = 2 * r->nf * up256(r->field_elems * sizeof(float));
    if (req->kind == STENCIL_MHD8) b += 16 * up256(r->ncell * sizeof(float));
    b += up256(sizeof(CUtensorMap) * 2 * r->nf);
    r->bytes = b;
    if ((int64_t)b > s->budget) {
        delete r;
        return sfail(s, STENCIL_EINVAL, "problem larger than the whole HBM budget");
    }
    cudaError_t e = cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) { delete r; return scuda(s, e, "cudaEventCreate"); }
    r->ticket = s->next_ticket++;
    s->table[r->ticket] = r;
    s->pending.push_back(r);
    *ticket = r->ticket;
    return STENCIL_OK;
}

stencil_status stencil_server_progress(stencil_server_t s, int *n_pending, int *n_active, int *n_done) {
    if (!s) return sfail(nullptr, STENCIL_EINVAL, "server is NULL");
    cudaStream_t st = s->stream;
    // 1. retire finished copy-backs
    for (size_t i = 0; i < s->completing.size();) {
        Req *r = s->completing[i];
        const cudaError_t q = cudaEventQuery(r->ev);
        if (q == cudaSuccess) {
            SCK(s, cudaFreeAsync(r->base, st), "pool free");
            r->base = nullptr;
            s->used -= (int64_t)r->bytes;
            r->state = ST_DONE;
            s->cell_updates += r->ncell * (int64_t)r->nsteps;
            s->completing[i] = s->completing.back();
            s->completing.pop_back();
        } else if (q == cudaErrorNotReady) {
            ++i;
        } else {
            return scuda(s, q, "completion event");
        }
    }
    // 2. admit in arrival order while budget and slots allow
    while (!s->pending.empty() && (int)(s->active.size() + s->completing.size()) < s->max_active &&
           s->used + (int64_t)s->pending.front()->bytes <= s->budget) {
        Req *r = s->pending.front();
        s->pending.pop_front();
        stencil_status stt = admit(s, r);
        if (stt != STENCIL_OK) return stt;
    }
    // 3. one step of every active problem
    if (!s->active.empty()) {
        const int i = s->tab_i;
        SCK(s, cudaEventSynchronize(s->tab_ev[i]), "table reuse");
        unsigned char *h = s->host_tab[i];
        BatchHeader *hdr = reinterpret_cast<BatchHeader *>(h);
        std::memset(hdr, 0, sizeof(BatchHeader));
        const size_t off_heat = up256(sizeof(BatchHeader));
        const size_t off_mhd = off_heat + up256(sizeof(BatchHeat) * s->max_active);
        const size_t mhd_stride = up256(sizeof(BatchMhd) * s->max_active);
        const size_t off_xc = off_mhd + 3 * mhd_stride;
        BatchHeat *hh = reinterpret_cast<BatchHeat *>(h + off_heat);
        BatchXcorr *hx = reinterpret_cast<BatchXcorr *>(h + off_xc);
        for (Req *r : s->active) {
            if (r->kind == STENCIL_DIFFUSION) {
                BatchHeat &it = hh[hdr->n_heat++];
                it.map = r->dmaps + r->cur;
                it.out = r->set[r->cur ^ 1][0];
                it.g = r->g;
                it.g0 = r->g0;
                std::memcpy(it.ga, r->ga, sizeof(it.ga));
                it.zc = r->zc;
                it.tiles_x = r->tiles[0];
                it.tiles_y = r->tiles[1];
                it.tiles_z = r->tiles[2];
                it.cta_begin = hdr->heat_ctas;
                hdr->heat_ctas += r->tiles[0] * r->tiles[1] * r->tiles[2];
            } else if (r->kind == STENCIL_MHD8) {
                for (int sub = 0; sub < 3; ++sub) {
                    BatchMhd &it = reinterpret_cast<BatchMhd *>(h + off_mhd + sub * mhd_stride)[hdr->n_mhd];
                    const int src = r->cur ^ (sub & 1);
                    it.maps = r->dmaps + src * 8;
                    for (int q = 0; q < 8; ++q) it.fout.p[q] = r->set[src ^ 1][q];
                    it.w = r->w;
                    it.kc = r->kc;
                    it.g = r->g;
                    it.k = r->k;
                    it.zc = r->zc;
                    it.tiles_x = r->tiles[0];
                    it.tiles_y = r->tiles[1];
                    it.tiles_z = r->tiles[2];
                    it.cta_begin = hdr->mhd_ctas;
                }
                hdr->n_mhd++;
                hdr->mhd_ctas += r->tiles[0] * r->tiles[1] * r->tiles[2];
            } else {
                BatchXcorr &it = hx[hdr->n_xc++];
                it.in = r->set[r->cur][0];
                it.out = r->set[r->cur ^ 1][0];
                it.g = r->g;
                std::memcpy(it.w, r->w7, sizeof(it.w));
                it.chunks = r->tiles[0];
                it.cta_begin = hdr->xc_ctas;
                hdr->xc_ctas += r->tiles[0];
            }
        }
        // upload the table region in use (header + every used item range), then every batched
        // launch, as one replay of the captured iteration graph
        const size_t used_bytes = hdr->n_xc ? off_xc + sizeof(BatchXcorr) * hdr->n_xc
                                  : hdr->n_mhd ? off_mhd + 2 * mhd_stride + sizeof(BatchMhd) * hdr->n_mhd
                                  : off_heat + sizeof(BatchHeat) * hdr->n_heat;
        SCK(s, cudaGraphExecMemcpyNodeSetParams1D(s->exec[i], s->copy_node[i], s->dev_tab, h, used_bytes,
                                                  cudaMemcpyHostToDevice),
            "table upload size");
        SCK(s, cudaGraphLaunch(s->exec[i], st), "batched iteration graph");
        SCK(s, cudaEventRecord(s->tab_ev[i], st), "table event");
        s->tab_i ^= 1;
        // 4. advance the bookkeeping; queue copy-back of finished problems
        for (size_t a = 0; a < s->active.size();) {
            Req *r = s->active[a];
            r->cur ^= 1;  // heat and xcorr: one pass; MHD: three substeps, also an odd count
            if (++r->steps_done == r->nsteps) {
                stencil_status stt = finish(s, r);
                if (stt != STENCIL_OK) return stt;
                s->active[a] = s->active.back();
                s->active.pop_back();
            } else {
                ++a;
            }
        }
    }
    if (n_pending) *n_pending = (int)s->pending.size();
    if (n_active) *n_active = (int)(s->active.size() + s->completing.size());
    if (n_done) {
        int d = 0;
        for (auto &kv : s->table) d += kv.second->state == ST_DONE;
        *n_done = d;
    }
    return STENCIL_OK;
}

const char *stencil_server_variant(stencil_server_t s, stencil_kind kind) {
    if (!s) return "?";
    if (kind == STENCIL_DIFFUSION) return diffusion_batch_shape_name(s->heat_shape);
    if (kind == STENCIL_MHD8) return mhd_batch_shape_name(s->mhd_shape);
    if (kind == STENCIL_XCORR) return "batch_chunk2184_one_sweep";
    return "?";
}

stencil_status stencil_server_poll(stencil_server_t s, int64_t ticket, int *state) {
    if (!s) return sfail(nullptr, STENCIL_EINVAL, "server is NULL");
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return sfail(s, STENCIL_EINVAL, "unknown ticket");
    if (state) *state = it->second->state;
    return STENCIL_OK;
}

stencil_status stencil_server_cancel(stencil_server_t s, int64_t ticket) {
    if (!s) return sfail(nullptr, STENCIL_EINVAL, "server is NULL");
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return sfail(s, STENCIL_EINVAL, "unknown ticket");
    Req *r = it->second;
    if (r->state == ST_PENDING) {
        for (auto p = s->pending.begin(); p != s->pending.end(); ++p)
            if (*p == r) {
                s->pending.erase(p);
                break;
            }
    } else if (r->state == ST_ACTIVE) {
        for (size_t a = 0; a < s->active.size(); ++a)
            if (s->active[a] == r) {
                s->active[a] = s->active.back();
                s->active.pop_back();
                break;
            }
        // the iteration already launched may still read the block: free it in stream order
        SCK(s, cudaFreeAsync(r->base, s->stream), "pool free");
        r->base = nullptr;
        s->used -= (int64_t)r->bytes;
    } else {
        return sfail(s, STENCIL_EINVAL, "ticket is already completing, done or cancelled");
    }
    r->state = ST_CANCELLED;
    for (int q = 0; q < 8; ++q) {
        r->host_in[q] = nullptr;
        r->host_out[q] = nullptr;
    }
    return STENCIL_OK;
}

stencil_status stencil_server_stats(stencil_server_t s, int64_t *bytes_in_use, int64_t *peak_bytes,
                                    int64_t *cell_updates_done) {
    if (!s) return sfail(nullptr, STENCIL_EINVAL, "server is NULL");
    if (bytes_in_use) *bytes_in_use = s->used;
    if (peak_bytes) *peak_bytes = s->peak;
    if (cell_updates_done) *cell_updates_done = s->cell_updates;
    return STENCIL_OK;
}

stencil_status stencil_server_sync(stencil_server_t s) {
    if (!s) return sfail(nullptr, STENCIL_EINVAL, "server is NULL");
    SCK(s, cudaStreamSynchronize(s->stream), "cudaStreamSynchronize");
    unsigned h = 0;
    SCK(s, cudaMemcpy(&h, s->err, sizeof(unsigned), cudaMemcpyDeviceToHost), "read error word");
    if (h) {
        SCK(s, cudaMemset(s->err, 0, sizeof(unsigned)), "clear error word");
        return sfail(s, STENCIL_ETIMEOUT, "a bounded wait expired in a batched kernel");
    }
    return STENCIL_OK;
}

const char *stencil_server_last_error_detail(stencil_server_t s) {
    return s ? s->detail.c_str() : g_server_detail.c_str();
}

}  // extern "C"
