// api.cu -- the C ABI of include/stencil.h: plans, layout, validation, scratch ownership,
// pass scheduling (ping-pong), TMA descriptor encoding and error reporting.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/stencil.h"
#include "internal.h"

using namespace stn;

namespace {

thread_local std::string g_create_detail;

struct TmaEntry {
    const void *ptr;
    int box[3];
    CUtensorMap map;
};

int esize_of(stencil_dtype t) {
    switch (t) {
    case STENCIL_I32: return 4;
    case STENCIL_F64: return 8;
    case STENCIL_F32: return 4;
    case STENCIL_BF16: return 2;
    }
    return 0;
}

const char *dtype_name(stencil_dtype t) {
    switch (t) {
    case STENCIL_I32: return "i32";
    case STENCIL_F64: return "f64";
    case STENCIL_F32: return "f32";
    case STENCIL_BF16: return "bf16";
    }
    return "?";
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

}  // namespace

struct stencil_plan {
    int device = 0;
    int ndim = 0, radius = 0, nfields = 0;
    stencil_kind kind = STENCIL_XCORR;
    stencil_bc bc = STENCIL_BC_PERIODIC;
    stencil_dtype storage = STENCIL_F64, compute = STENCIL_F64;
    stencil_params par{};
    Geom geom{};
    int esize = 0;
    int64_t bytes_per_field = 0;
    // coefficients
    int32_t gi[9] = {};
    double gd[65] = {};  // FP64 radius <= 4; FP32 radius <= 32 (the temporally blocked kernel)
    float gf[65] = {};
    DiffCoef dcoef{};
    MhdConst mconst{};
    // library-owned scratch
    void *tmp[8] = {};  // second field set for ping-pong (padded layout)
    void *w[8] = {};    // MHD8: w[0] the RK register (dense interior, storage type, 8 fields
    void *kc[8] = {};   // interleaved per cell); kc[0] the Kahan terms, same layout
    double *partials = nullptr;
    double *red_out = nullptr;
    unsigned *err = nullptr;
    void *wdev = nullptr;  // XCORR of radius > 4: the 2r+1 weights on the device (storage type)
    unsigned long long *psync = nullptr;  // sync words of the persistent heat schedule (persist.cuh)
    int64_t psync_words = 0;
    int variant = 0;
    int zmode = 0;           // z-chunk length mode of the streaming kernels (zchunk_len)
    int tuned_from_cache = 0;
    float tuned_ms = 0.f;
    std::vector<TmaEntry> tma;
    std::string detail;
};

static stencil_status fail(stencil_t p, stencil_status st, const std::string &msg) {
    if (p) p->detail = msg;
    else g_create_detail = msg;
    return st;
}

static stencil_status cuda_fail(stencil_t p, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    cudaGetLastError();  // clear the sticky non-fatal error state
    return fail(p, e == cudaErrorMemoryAllocation ? STENCIL_ENOMEM : STENCIL_ECUDA, m);
}

#define CK(p, call, what)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(p, e_, what); \
    } while (0)

static stencil_status check_device(stencil_t p) {
    int d = -1;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaGetDevice");
    if (d != p->device)
        return fail(p, STENCIL_EINVAL, "plan belongs to device " + std::to_string(p->device) +
                                           " but device " + std::to_string(d) + " is current");
    return STENCIL_OK;
}

static int storage_code(stencil_dtype t) {
    switch (t) {
    case STENCIL_I32: return 0;
    case STENCIL_F64: return 1;
    case STENCIL_F32: return 2;
    case STENCIL_BF16: return 3;
    }
    return -1;
}

static void free_scratch(stencil_t p) {
    for (int q = 0; q < 8; ++q) {
        if (p->tmp[q]) cudaFree(p->tmp[q]);
        if (p->w[q]) cudaFree(p->w[q]);
        if (p->kc[q]) cudaFree(p->kc[q]);
        p->tmp[q] = p->w[q] = p->kc[q] = nullptr;
    }
    if (p->partials) cudaFree(p->partials);
    if (p->red_out) cudaFree(p->red_out);
    if (p->err) cudaFree(p->err);
    if (p->wdev) cudaFree(p->wdev);
    if (p->psync) cudaFree(p->psync);
    p->psync = nullptr;
    p->psync_words = 0;
    p->partials = p->red_out = nullptr;
    p->err = nullptr;
    p->wdev = nullptr;
}

// Encode (or fetch from the per-plan cache) the TMA descriptor of a field for a box shape.
static stencil_status tma_map(stencil_t p, const void *ptr, const int box[3], CUtensorMap *out) {
    for (auto &e : p->tma)
        if (e.ptr == ptr && e.box[0] == box[0] && e.box[1] == box[1] && e.box[2] == box[2]) {
            *out = e.map;
            return STENCIL_OK;
        }
    auto fn = encode_fn();
    if (!fn) return fail(p, STENCIL_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
    CUtensorMapDataType dt;
    switch (p->storage) {
    case STENCIL_F64: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT64; break;
    case STENCIL_F32: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
    case STENCIL_BF16: dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
    default: dt = CU_TENSOR_MAP_DATA_TYPE_INT32; break;
    }
    const Geom &g = p->geom;
    cuuint64_t dims[3] = {(cuuint64_t)g.pad[0], (cuuint64_t)g.pad[1], (cuuint64_t)g.pad[2]};
    cuuint64_t strides[2] = {(cuuint64_t)(g.pad[0] * p->esize), (cuuint64_t)(g.pad[0] * g.pad[1] * p->esize)};
    cuuint32_t bx[3] = {(cuuint32_t)box[0], (cuuint32_t)box[1], (cuuint32_t)box[2]};
    cuuint32_t es[3] = {1, 1, 1};
    TmaEntry ent;
    ent.ptr = ptr;
    std::memcpy(ent.box, box, sizeof(ent.box));
    CUresult r = fn(&ent.map, dt, 3, const_cast<void *>(ptr), dims, strides, bx, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(p, STENCIL_ECUDA, "cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r));
    if (p->tma.size() >= 96) p->tma.erase(p->tma.begin());
    p->tma.push_back(ent);
    *out = ent.map;
    return STENCIL_OK;
}

static stencil_status check_ptrs(stencil_t p, void *const *f, const char *what) {
    if (!f) return fail(p, STENCIL_EINVAL, std::string(what) + " is NULL");
    for (int q = 0; q < p->nfields; ++q) {
        if (!f[q]) return fail(p, STENCIL_EINVAL, std::string(what) + "[" + std::to_string(q) + "] is NULL");
        if (reinterpret_cast<uintptr_t>(f[q]) % 16 != 0)
            return fail(p, STENCIL_EINVAL, std::string(what) + "[" + std::to_string(q) + "] is not 16-byte aligned");
    }
    return STENCIL_OK;
}

static Ptrs8 ptrs(void *const *f, int n) {
    Ptrs8 r{};
    for (int q = 0; q < n; ++q) r.p[q] = f[q];
    return r;
}

// ------------------------------------------------------------------ autotuning cache
// Winners of stencil_autotune, kept for the life of the process and, when the environment
// variable STENCIL_AUTOTUNE_CACHE names a file, in that file: one line per problem class,
// "key <TAB> variant name <TAB> z-chunk mode <TAB> ms".  The key holds the GPU's name and SM
// count, the kind, storage, radius, boundary, dims and steps per call, so a choice is reused only
// for the same problem on the same kind of GPU.  Later lines win; a damaged line is skipped.
namespace {
struct TuneRec {
    std::string variant;
    int zmode = 0;
    float ms = 0.f;
};
std::mutex g_tune_mu;
std::map<std::string, TuneRec> g_tune;
std::map<std::string, std::string> g_tune_last;  // problem-class prefix (no dims / steps) -> last winner
std::string g_tune_loaded;                       // path whose lines are in g_tune

void tune_put_locked(const std::string &key, const TuneRec &rec) {
    g_tune[key] = rec;
    const size_t cut = key.find("|d3:");
    if (cut != std::string::npos) g_tune_last[key.substr(0, cut + 4)] = rec.variant;
}

std::string tune_path() {
    const char *e = std::getenv("STENCIL_AUTOTUNE_CACHE");
    return e ? std::string(e) : std::string();
}

void tune_load_locked(const std::string &path) {
    if (path.empty() || path == g_tune_loaded) return;
    g_tune_loaded = path;
    std::ifstream in(path);
    std::string line;
    while (std::getline(in, line)) {
        std::istringstream ls(line);
        std::string key, var, zm, ms;
        if (!std::getline(ls, key, '\t') || !std::getline(ls, var, '\t') || !std::getline(ls, zm, '\t') ||
            !std::getline(ls, ms))
            continue;
        char *end = nullptr;
        const long z = std::strtol(zm.c_str(), &end, 10);
        if (end == zm.c_str() || z < 0 || z >= ZMODES || var.empty()) continue;
        tune_put_locked(key, TuneRec{var, (int)z, std::strtof(ms.c_str(), nullptr)});
    }
}

std::string gpu_tag(int dev) {
    static std::string tags[64];
    if (dev < 0 || dev >= 64) return "gpu?";
    if (tags[dev].empty()) {
        cudaDeviceProp pr{};
        if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return "gpu?";
        std::string n = pr.name;
        for (auto &ch : n)
            if (ch == '\t' || ch == ' ') ch = '_';
        tags[dev] = n + "_sm" + std::to_string(pr.multiProcessorCount);
    }
    return tags[dev];
}
}  // namespace

namespace stn {
int tuned_batch_shape(int kind) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    const std::string pref = gpu_tag(dev) + "|k" + std::to_string(kind) + "|s" + std::to_string((int)STENCIL_F32) +
                             "|r3|bc" + std::to_string((int)STENCIL_BC_PERIODIC) + "|d3:";
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load_locked(tune_path());
    auto it = g_tune_last.find(pref);
    if (it == g_tune_last.end()) return -1;
    // the batched shapes: heat 0 = 4 warps x 2 rows, 1 = 8 warps x 2 rows; MHD 0 = 32 x 4 with
    // two CTAs per SM, 1 = 32 x 8 with one
    const std::string &v = it->second;
    if (kind == STENCIL_DIFFUSION) return v.find("by8") != std::string::npos ? 1 : 0;
    return v.find("_b1") != std::string::npos ? 1 : 0;
}
}  // namespace stn

static std::string tune_key(stencil_t p, int nsteps) {
    std::ostringstream k;
    k << gpu_tag(p->device) << "|k" << (int)p->kind << "|s" << (int)p->storage << "|r" << p->radius << "|bc"
      << (int)p->bc << "|d" << p->ndim << ":" << p->geom.n[0] << "x" << p->geom.n[1] << "x" << p->geom.n[2] << "|n"
      << nsteps;
    return k.str();
}

extern "C" {

static stencil_status read_err(stencil_t p, cudaStream_t s);

int stencil_abi_version(void) { return STENCIL_ABI_VERSION; }

const char *stencil_strerror(stencil_status s) {
    switch (s) {
    case STENCIL_OK: return "STENCIL_OK";
    case STENCIL_EINVAL: return "STENCIL_EINVAL: invalid argument";
    case STENCIL_ENOMEM: return "STENCIL_ENOMEM: out of memory";
    case STENCIL_ECUDA: return "STENCIL_ECUDA: CUDA error";
    case STENCIL_EUNSUPPORTED: return "STENCIL_EUNSUPPORTED: combination not implemented";
    case STENCIL_ETIMEOUT: return "STENCIL_ETIMEOUT: bounded device wait expired";
    }
    return "unknown stencil_status";
}

const char *stencil_last_error_detail(stencil_t p) {
    return p ? p->detail.c_str() : g_create_detail.c_str();
}

// Centred 2nd-derivative weights of order 2r on points -r..r (unit spacing): c[0] for the centre,
// c[k] for each point at +-k; c_k = 2 (-1)^(k+1) (r!)^2 / (k^2 (r-k)! (r+k)!), c_0 = -2 sum 1/k^2.
static void central_d2_weights(int r, double *c) {
    auto fact = [](int k) {
        double f = 1.0;
        for (int i = 2; i <= k; ++i) f *= i;
        return f;
    };
    c[0] = 0.0;
    for (int k = 1; k <= r; ++k) {
        c[k] = ((k & 1) ? 2.0 : -2.0) * fact(r) * fact(r) / ((double)k * k * fact(r - k) * fact(r + k));
        c[0] -= 2.0 / ((double)k * k);
    }
}

stencil_status stencil_create(int ndim, const int64_t dims[3], int radius, const void *coeffs,
                              int ncoeffs, int nfields, stencil_bc bc, stencil_kind kind,
                              stencil_dtype storage, stencil_dtype compute,
                              const stencil_params *params, stencil_t *out) {
    g_create_detail.clear();
    if (!out) return fail(nullptr, STENCIL_EINVAL, "out is NULL");
    *out = nullptr;
    if (!dims) return fail(nullptr, STENCIL_EINVAL, "dims is NULL");
    if ((int)kind < 0 || (int)kind > 3) return fail(nullptr, STENCIL_EINVAL, "unknown kind");
    if ((int)bc < 0 || (int)bc > 2) return fail(nullptr, STENCIL_EINVAL, "unknown boundary condition");
    if (bc == STENCIL_BC_PERIODIC_XY && (ndim != 3 || (kind != STENCIL_DIFFUSION && kind != STENCIL_MHD8)))
        return fail(nullptr, STENCIL_EUNSUPPORTED, "STENCIL_BC_PERIODIC_XY needs a 3D DIFFUSION or MHD8 plan");
    if ((int)storage < 0 || (int)storage > 3 || (int)compute < 0 || (int)compute > 3)
        return fail(nullptr, STENCIL_EINVAL, "unknown dtype");
    if (ndim < 1 || ndim > 3) return fail(nullptr, STENCIL_EINVAL, "ndim must be 1, 2 or 3");
    for (int a = 0; a < ndim; ++a)
        if (dims[a] < 1 || dims[a] > (int64_t)1 << 31)
            return fail(nullptr, STENCIL_EINVAL, "dims[" + std::to_string(a) + "] out of range");
    if (radius < 0) return fail(nullptr, STENCIL_EINVAL, "radius must be >= 0");

    // kind-specific rules
    if (kind == STENCIL_XCORR) {
        if (ndim != 1) return fail(nullptr, STENCIL_EUNSUPPORTED, "XCORR supports ndim = 1");
        if (radius > 1024) return fail(nullptr, STENCIL_EUNSUPPORTED, "XCORR supports radius 0..1024");
        if (ncoeffs != 2 * radius + 1 || !coeffs)
            return fail(nullptr, STENCIL_EINVAL, "XCORR needs 2*radius+1 coefficients");
        if (nfields != 1) return fail(nullptr, STENCIL_EINVAL, "XCORR needs nfields = 1");
        if (storage != compute || storage == STENCIL_BF16)
            return fail(nullptr, STENCIL_EUNSUPPORTED, "XCORR supports I32/I32, F64/F64, F32/F32");
        if (radius > 4 && storage == STENCIL_I32)
            return fail(nullptr, STENCIL_EUNSUPPORTED, "XCORR of radius > 4 supports F64/F64 and F32/F32");
    } else if (kind == STENCIL_MAXFILTER) {
        if (ndim != 1) return fail(nullptr, STENCIL_EUNSUPPORTED, "MAXFILTER supports ndim = 1");
        if (radius > 1024) return fail(nullptr, STENCIL_EUNSUPPORTED, "MAXFILTER supports radius 0..1024");
        if (ncoeffs != 0) return fail(nullptr, STENCIL_EINVAL, "MAXFILTER takes no coefficients");
        if (nfields != 1) return fail(nullptr, STENCIL_EINVAL, "MAXFILTER needs nfields = 1");
        if (storage != compute || storage == STENCIL_BF16)
            return fail(nullptr, STENCIL_EUNSUPPORTED, "MAXFILTER supports I32/I32, F64/F64, F32/F32");
    } else {
        if (kind == STENCIL_DIFFUSION && (radius < 1 || radius > 4))
            return fail(nullptr, STENCIL_EUNSUPPORTED, "DIFFUSION supports radius 1..4");
        if (kind == STENCIL_MHD8 && radius != 3) return fail(nullptr, STENCIL_EINVAL, "MHD8 uses radius 3");
        if (ncoeffs != 0) return fail(nullptr, STENCIL_EINVAL, "DIFFUSION and MHD8 take no coefficients");
        if (!params) return fail(nullptr, STENCIL_EINVAL, "params is NULL");
        if (kind == STENCIL_MHD8 && ndim != 3) return fail(nullptr, STENCIL_EUNSUPPORTED, "MHD8 supports ndim = 3");
        for (int a = 0; a < ndim; ++a)
            if (!(params->dx[a] > 0.0) || !std::isfinite(params->dx[a]))
                return fail(nullptr, STENCIL_EINVAL, "grid spacing must be positive and finite");
        if (!std::isfinite(params->dt)) return fail(nullptr, STENCIL_EINVAL, "dt must be finite");
        if (kind == STENCIL_DIFFUSION) {
            if (nfields != 1) return fail(nullptr, STENCIL_EINVAL, "DIFFUSION needs nfields = 1");
            if (!((storage == STENCIL_F64 && compute == STENCIL_F64) ||
                  (storage == STENCIL_F32 && compute == STENCIL_F32)))
                return fail(nullptr, STENCIL_EUNSUPPORTED, "DIFFUSION supports F64/F64 and F32/F32");
        } else {
            if (nfields != 8) return fail(nullptr, STENCIL_EINVAL, "MHD8 needs nfields = 8");
            if (bc == STENCIL_BC_CALLER)
                return fail(nullptr, STENCIL_EUNSUPPORTED,
                            "MHD8 supports periodic boundaries (or periodic x/y with a caller z halo)");
            if (!((storage == STENCIL_F64 && compute == STENCIL_F64) ||
                  (storage == STENCIL_F32 && compute == STENCIL_F32) ||
                  (storage == STENCIL_BF16 && compute == STENCIL_F32)))
                return fail(nullptr, STENCIL_EUNSUPPORTED, "MHD8 supports F64/F64, F32/F32, BF16/F32");
            if (!(params->cp > 0.0) || !(params->gamma > 1.0) || !(params->mu0 > 0.0))
                return fail(nullptr, STENCIL_EINVAL, "MHD8 needs cp > 0, gamma > 1, mu0 > 0");
            if (!(params->K >= 0.0) || !std::isfinite(params->K))
                return fail(nullptr, STENCIL_EINVAL, "MHD8 needs a finite heat conductivity K >= 0");
        }
    }
    if (bc == STENCIL_BC_PERIODIC)
        for (int a = 0; a < ndim; ++a)
            if (dims[a] < 2 * radius + 1)
                return fail(nullptr, STENCIL_EINVAL, "periodic extents must be >= 2*radius+1");
    if (bc == STENCIL_BC_PERIODIC_XY) {
        if (dims[0] < 2 * radius + 1 || dims[1] < 2 * radius + 1)
            return fail(nullptr, STENCIL_EINVAL, "periodic extents must be >= 2*radius+1");
        if (dims[2] < radius)
            return fail(nullptr, STENCIL_EINVAL, "a z-slab needs at least radius planes");
    }

    stencil_plan *p = new (std::nothrow) stencil_plan;
    if (!p) return fail(nullptr, STENCIL_ENOMEM, "host allocation of the plan failed");
    p->ndim = ndim;
    p->radius = radius;
    p->nfields = nfields;
    p->kind = kind;
    p->bc = bc;
    p->storage = storage;
    p->compute = compute;
    if (params) p->par = *params;
    p->esize = esize_of(storage);

    // layout: x origin rounded up to 16 bytes, row pitch to 32 bytes
    const int v16 = 16 / p->esize;
    const int64_t xoff = ((radius + v16 - 1) / v16) * v16;
    const int64_t align32 = 32 / p->esize;
    Geom &g = p->geom;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = a < ndim ? dims[a] : 1;
        g.off[a] = (a == 0) ? xoff : (a < ndim ? radius : 0);
    }
    g.pad[0] = ((xoff + g.n[0] + xoff + align32 - 1) / align32) * align32;
    g.pad[1] = ndim >= 2 ? g.n[1] + 2 * radius : 1;
    g.pad[2] = ndim >= 3 ? g.n[2] + 2 * radius : 1;
    p->bytes_per_field = g.pad[0] * g.pad[1] * g.pad[2] * p->esize;

    // coefficients / constants
    std::vector<double> wide_w;  // XCORR radius > 4: weights copied to the device below
    if (kind == STENCIL_XCORR && radius > 4) {
        wide_w.assign(static_cast<const double *>(coeffs), static_cast<const double *>(coeffs) + ncoeffs);
        if (radius <= 32)  // FP32 radius 5..32 also runs the temporally blocked kernel
            for (int j = 0; j < ncoeffs; ++j) p->gf[j] = (float)wide_w[j];
    } else if (kind == STENCIL_MAXFILTER) {
    } else if (kind == STENCIL_XCORR) {
        for (int j = 0; j < ncoeffs; ++j) {
            if (storage == STENCIL_I32) p->gi[j] = static_cast<const int32_t *>(coeffs)[j];
            else {
                p->gd[j] = static_cast<const double *>(coeffs)[j];
                p->gf[j] = (float)p->gd[j];
            }
        }
    } else {
        static const double W1[3] = {3.0 / 4.0, -3.0 / 20.0, 1.0 / 60.0};
        static const double W2C = -49.0 / 18.0;
        static const double W2[3] = {3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0};
        static const double WM[3] = {270.0, -27.0, 2.0};
        const double *h = params->dx;
        if (kind == STENCIL_DIFFUSION) {
            // Eq. 5/7: g = c1 + dt alpha (sum over the ndim axes of the order-2r Laplacian)
            double c2[5];
            central_d2_weights(radius, c2);
            const double s = params->dt * params->alpha;
            double g0 = 1.0;
            p->dcoef = DiffCoef{};
            p->dcoef.r = radius;
            for (int a = 0; a < ndim; ++a) {
                g0 += s * c2[0] / (h[a] * h[a]);
                for (int i = 0; i < radius; ++i) p->dcoef.ga[a][i] = s * c2[i + 1] / (h[a] * h[a]);
            }
            p->dcoef.g0 = g0;
            if (ndim == 1) {  // 1D: the folded step is the cross-correlation of Eq. 3 with these weights
                for (int j = -radius; j <= radius; ++j) {
                    const double w = j == 0 ? g0 : p->dcoef.ga[0][std::abs(j) - 1];
                    p->gd[j + radius] = w;
                    p->gf[j + radius] = (float)w;
                }
            }
        } else {
            MhdConst &c = p->mconst;
            for (int a = 0; a < 3; ++a) {
                c.d2c[a] = W2C / (h[a] * h[a]);
                for (int i = 0; i < 3; ++i) {
                    c.d1[a][i] = W1[i] / h[a];
                    c.d2[a][i] = W2[i] / (h[a] * h[a]);
                }
            }
            const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
            for (int pi = 0; pi < 3; ++pi)
                for (int i = 0; i < 3; ++i)
                    c.dm[pi][i] = WM[i] / (720.0 * h[pairs[pi][0]] * h[pairs[pi][1]]);
            c.cs0sq = params->cs0 * params->cs0;
            c.gamma = params->gamma;
            c.inv_cp = 1.0 / params->cp;
            c.lnrho0 = params->lnrho0;
            c.nu = params->nu;
            c.eta = params->eta;
            c.zeta = params->zeta;
            c.mu0 = params->mu0;
            c.inv_mu0 = 1.0 / params->mu0;
            c.cp_gm1 = params->cp * (params->gamma - 1.0);
            c.K = params->K;
            c.dt = params->dt;
        }
    }

    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        stencil_status st = cuda_fail(nullptr, e, "cudaGetDevice");
        delete p;
        return st;
    }
    // scratch
    auto alloc = [&](void **dst, size_t bytes, const char *what) -> bool {
        cudaError_t ee = cudaMalloc(dst, bytes);
        if (ee != cudaSuccess) {
            cuda_fail(nullptr, ee, what);
            *dst = nullptr;
            return false;
        }
        return true;
    };
    bool okay = true;
    const size_t ncell = (size_t)(g.n[0] * g.n[1] * g.n[2]);
    for (int q = 0; q < nfields && okay; ++q) okay = alloc(&p->tmp[q], p->bytes_per_field, "cudaMalloc(ping-pong field)");
    if (kind == STENCIL_MHD8) {
        okay = alloc(&p->w[0], 8 * ncell * p->esize, "cudaMalloc(RK register)");
        if (okay && storage != STENCIL_F64) okay = alloc(&p->kc[0], 8 * ncell * p->esize, "cudaMalloc(Kahan terms)");
    }
    if (okay) okay = alloc((void **)&p->partials, sizeof(double) * norms_blocks() * nfields * 4, "cudaMalloc(norm partials)");
    if (okay) okay = alloc((void **)&p->red_out, sizeof(double) * nfields * 4, "cudaMalloc(norm result)");
    if (okay) okay = alloc((void **)&p->err, sizeof(unsigned), "cudaMalloc(error word)");
    if (okay && !wide_w.empty()) {
        okay = alloc(&p->wdev, wide_w.size() * p->esize, "cudaMalloc(weights)");
        if (okay) {
            std::vector<float> wf(wide_w.begin(), wide_w.end());
            const void *src = storage == STENCIL_F64 ? (const void *)wide_w.data() : (const void *)wf.data();
            e = cudaMemcpy(p->wdev, src, wide_w.size() * p->esize, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) { cuda_fail(nullptr, e, "cudaMemcpy(weights)"); okay = false; }
        }
    }
    if (okay) {
        e = cudaMemset(p->err, 0, sizeof(unsigned));
        if (e != cudaSuccess) { cuda_fail(nullptr, e, "cudaMemset(error word)"); okay = false; }
    }
    if (!okay) {
        stencil_status st = g_create_detail.find("cudaErrorMemoryAllocation") != std::string::npos ? STENCIL_ENOMEM : STENCIL_ECUDA;
        free_scratch(p);
        delete p;
        return st;
    }
    *out = p;
    return STENCIL_OK;
}

void stencil_destroy(stencil_t p) {
    if (!p) return;
    cudaDeviceSynchronize();
    free_scratch(p);
    delete p;
}

stencil_status stencil_layout(stencil_t p, int64_t padded[3], int64_t pitch[3], int64_t origin[3],
                              int64_t *bytes_per_field) {
    if (!p) return fail(nullptr, STENCIL_EINVAL, "plan is NULL");
    const Geom &g = p->geom;
    for (int a = 0; a < 3; ++a) {
        if (padded) padded[a] = g.pad[a];
        if (origin) origin[a] = g.off[a];
    }
    if (pitch) {
        pitch[0] = 1;
        pitch[1] = g.pad[0];
        pitch[2] = g.pad[0] * g.pad[1];
    }
    if (bytes_per_field) *bytes_per_field = p->bytes_per_field;
    return STENCIL_OK;
}

stencil_status stencil_halo_fill(stencil_t p, void *const *fields, void *stream) {
    if (!p) return fail(nullptr, STENCIL_EINVAL, "plan is NULL");
    stencil_status st = check_device(p);
    if (st != STENCIL_OK) return st;
    if ((st = check_ptrs(p, fields, "fields")) != STENCIL_OK) return st;
    if (p->bc == STENCIL_BC_CALLER) return STENCIL_OK;
    CK(p, launch_halo_fill(p->geom, p->radius, p->esize, ptrs(fields, p->nfields), p->nfields,
                           (cudaStream_t)stream, p->bc == STENCIL_BC_PERIODIC),
       "halo_fill launch");
    return STENCIL_OK;
}

// XCORR plans that run the temporally blocked, register-window kernel (csrc/xcorr.cu): radius
// <= 4, and FP32 up to radius 32 (it beats the wide kernel there); the rest run the wide kernel.
static bool xcorr_blocked(stencil_t p) {
    return p->kind == STENCIL_XCORR && (p->radius <= 4 || (p->storage == STENCIL_F32 && p->radius <= 32));
}

// One pass of the plan's kernel from src to dst (sub = RK substep for MHD8).
static stencil_status run_pass(stencil_t p, void *const *src, void *const *dst, int sweeps, int sub,
                               cudaStream_t s) {
    const bool periodic = p->bc == STENCIL_BC_PERIODIC;
    const Geom &g = p->geom;
    if (p->kind == STENCIL_MAXFILTER) {
        CK(p, launch_maxfilter(storage_code(p->storage), p->radius, src[0], dst[0], g, periodic, periodic, p->err, s),
           "maxfilter launch");
        return STENCIL_OK;
    }
    if (p->kind == STENCIL_XCORR && !xcorr_blocked(p)) {
        CK(p, launch_xcorr_wide(storage_code(p->storage), p->radius, src[0], dst[0], g, p->wdev, periodic, periodic,
                                p->err, s),
           "xcorr (wide) launch");
        return STENCIL_OK;
    }
    if (p->kind == STENCIL_XCORR) {
        const void *cf = p->storage == STENCIL_I32 ? (const void *)p->gi
                         : p->storage == STENCIL_F64 ? (const void *)p->gd : (const void *)p->gf;
        CK(p, launch_xcorr(storage_code(p->storage), p->radius, src[0], dst[0], g, cf, sweeps, periodic,
                           periodic, s),
           "xcorr launch");
        return STENCIL_OK;
    }
    if (p->kind == STENCIL_DIFFUSION && p->ndim == 1) {  // folded weights through the XCORR kernel
        const void *cf = p->storage == STENCIL_F64 ? (const void *)p->gd : (const void *)p->gf;
        CK(p, launch_xcorr(storage_code(p->storage), p->radius, src[0], dst[0], g, cf, sweeps, periodic, periodic, s),
           "diffusion (1D) launch");
        return STENCIL_OK;
    }
    if (p->kind == STENCIL_DIFFUSION && p->ndim == 2 && sweeps > 1) {  // temporally blocked pass
        CK(p, launch_diffusion2d_tb(storage_code(p->storage), sweeps, src[0], dst[0], g, p->dcoef, s),
           "diffusion (2D, temporally blocked) launch");
        return STENCIL_OK;
    }
    if (p->kind == STENCIL_DIFFUSION) {
        int box[3];
        if (p->ndim == 2) diffusion2d_box(storage_code(p->storage), p->radius, box);
        else diffusion_box(storage_code(p->storage), p->radius, p->variant, box);
        CUtensorMap m;
        stencil_status st = tma_map(p, src[0], box, &m);
        if (st != STENCIL_OK) return st;
        if (p->ndim == 2)
            CK(p, launch_diffusion2d(storage_code(p->storage), &m, dst[0], g, p->dcoef, periodic, p->err, s),
               "diffusion (2D) launch");
        else
            CK(p, launch_diffusion(storage_code(p->storage), &m, dst[0], g, p->dcoef, p->bc != STENCIL_BC_CALLER,
                                   p->err, s, p->variant, p->zmode),
               "diffusion launch");
        return STENCIL_OK;
    }
    int box[3];
    mhd_box(storage_code(p->storage), p->variant, box);
    MhdMaps maps;
    for (int q = 0; q < 8; ++q) {
        stencil_status st = tma_map(p, src[q], box, &maps.m[q]);
        if (st != STENCIL_OK) return st;
    }
    Ptrs8 none{};
    CK(p, launch_mhd(storage_code(p->storage), 0, sub, maps, ptrs(dst, 8), p->w[0], p->kc[0], none,
                     g, p->mconst, true, p->err, s, p->variant, p->zmode),
       "mhd launch");
    return STENCIL_OK;
}

// All nsteps steps of a 3D heat plan whose variant has the persistent schedule: one halo fill
// of the input, then one cooperative launch.  The plan's sync words grow to the launch's unit
// count on first use (not while the stream is being captured into a graph).
static stencil_status step_persistent(stencil_t p, void *const *fin, void *const *fout, int nsteps,
                                      cudaStream_t s) {
    const int dt = storage_code(p->storage);
    int64_t units = 0;
    CK(p, launch_diffusion_persist(dt, nullptr, nullptr, nullptr, p->geom, p->dcoef, false, nsteps, nullptr, 0,
                                   p->err, s, p->variant, p->zmode, &units),
       "persistent heat schedule (unit count)");
    const int64_t need = PERSIST_HDR + units;
    if (need > p->psync_words) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        CK(p, cudaStreamIsCapturing(s, &cap), "cudaStreamIsCapturing");
        if (cap != cudaStreamCaptureStatusNone)
            return fail(p, STENCIL_EINVAL,
                        "the persistent schedule allocates its sync words on first use: run it once before "
                        "capturing it into a graph");
        CK(p, cudaStreamSynchronize(s), "cudaStreamSynchronize");
        if (p->psync) cudaFree(p->psync);
        p->psync = nullptr;
        p->psync_words = 0;
        CK(p, cudaMalloc(&p->psync, need * sizeof(unsigned long long)), "cudaMalloc (sync words)");
        CK(p, cudaMemsetAsync(p->psync, 0, need * sizeof(unsigned long long), s), "cudaMemsetAsync (sync words)");
        p->psync_words = need;
    }
    if (p->bc != STENCIL_BC_CALLER)
        CK(p, launch_halo_fill(p->geom, p->radius, p->esize, ptrs(fin, 1), 1, s, p->bc == STENCIL_BC_PERIODIC),
           "halo_fill launch");
    int box[3];
    diffusion_box(dt, p->radius, p->variant, box);
    CUtensorMap maps[3];
    const void *bufs[3] = {fin[0], p->tmp[0], fout[0]};
    for (int i = 0; i < 3; ++i) {
        stencil_status st = tma_map(p, bufs[i], box, &maps[i]);
        if (st != STENCIL_OK) return st;
    }
    CK(p, launch_diffusion_persist(dt, maps, p->tmp[0], fout[0], p->geom, p->dcoef, p->bc != STENCIL_BC_CALLER,
                                   nsteps, p->psync, p->psync_words, p->err, s, p->variant, p->zmode, &units),
       "persistent heat launch");
    return STENCIL_OK;
}

stencil_status stencil_step(stencil_t p, void *const *fin, void *const *fout, int nsteps, void *stream) {
    if (!p) return fail(nullptr, STENCIL_EINVAL, "plan is NULL");
    stencil_status st = check_device(p);
    if (st != STENCIL_OK) return st;
    if ((st = check_ptrs(p, fin, "fields_in")) != STENCIL_OK) return st;
    if ((st = check_ptrs(p, fout, "fields_out")) != STENCIL_OK) return st;
    for (int q = 0; q < p->nfields; ++q)
        for (int r = 0; r < p->nfields; ++r)
            if (fin[q] == fout[r]) return fail(p, STENCIL_EINVAL, "fields_in and fields_out alias");
    if (nsteps < 0) return fail(p, STENCIL_EINVAL, "nsteps must be >= 0");
    const bool periodic = p->bc == STENCIL_BC_PERIODIC;
    if (p->bc == STENCIL_BC_PERIODIC_XY && p->kind == STENCIL_MHD8)
        return fail(p, STENCIL_EINVAL, "an MHD8 z-slab advances one RK substep per call (stencil_substep)");
    if (!periodic && nsteps != 1)
        return fail(p, STENCIL_EINVAL, "caller-filled boundaries allow exactly one step per call");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t ncell = (size_t)(p->geom.n[0] * p->geom.n[1] * p->geom.n[2]);
    if (nsteps == 0) {
        for (int q = 0; q < p->nfields; ++q)
            CK(p, cudaMemcpyAsync(fout[q], fin[q], p->bytes_per_field, cudaMemcpyDeviceToDevice, s), "copy");
        return stencil_halo_fill(p, fout, stream);
    }

    if (p->kind == STENCIL_DIFFUSION && p->ndim == 3 &&
        diffusion_persistent(storage_code(p->storage), p->radius, p->variant))
        return step_persistent(p, fin, fout, nsteps, s);

    // pass list
    std::vector<int> sweeps;  // XCORR (and 1D DIFFUSION): sweeps per launch; others: one entry per pass
    int npass;
    const bool xcorr_like = p->kind == STENCIL_XCORR || p->kind == STENCIL_MAXFILTER ||
                            (p->kind == STENCIL_DIFFUSION && p->ndim == 1);
    if (xcorr_like) {
        // temporal blocking for the radius <= 4 kernel; one sweep per launch otherwise
        const bool single = !periodic || p->kind == STENCIL_MAXFILTER || (p->kind == STENCIL_XCORR && !xcorr_blocked(p));
        const int maxs = single ? 1 : xcorr_max_sweeps_per_launch(p->radius);
        for (int left = nsteps; left > 0;) {
            int k = std::min(left, maxs);
            sweeps.push_back(k);
            left -= k;
        }
        npass = (int)sweeps.size();
    } else if (p->kind == STENCIL_DIFFUSION && p->ndim == 2 && p->variant > 0 && periodic &&
               diffusion2d_tb_ok(storage_code(p->storage), p->geom)) {
        // temporal blocking: passes of K = 2 or 4 steps, the remainder one step at a time
        const int k = p->variant == 1 ? 2 : 4;
        for (int left = nsteps; left > 0;) {
            const int take = left >= k ? k : 1;
            sweeps.push_back(take);
            left -= take;
        }
        npass = (int)sweeps.size();
    } else {
        npass = p->kind == STENCIL_MHD8 ? 3 * nsteps : nsteps;
        sweeps.assign(npass, 1);
    }
    if (p->bc != STENCIL_BC_CALLER && !xcorr_like)
        CK(p, launch_halo_fill(p->geom, p->radius, p->esize, ptrs(fin, p->nfields), p->nfields, s, periodic),
           "halo_fill launch");
    if (p->kind == STENCIL_MHD8 && p->storage != STENCIL_F64)
        CK(p, cudaMemsetAsync(p->kc[0], 0, 8 * ncell * p->esize, s), "clear Kahan terms");

    // ping-pong so that the last pass writes fields_out and fields_in is only read
    void *const *src = fin;
    for (int i = 1; i <= npass; ++i) {
        void *const *dst = ((npass - i) % 2 == 0) ? fout : (void *const *)p->tmp;
        st = run_pass(p, src, dst, sweeps[i - 1], (i - 1) % 3, s);
        if (st != STENCIL_OK) return st;
        src = dst;
    }
    return STENCIL_OK;
}

stencil_status stencil_step_host(stencil_t p, const void *const *host_in, void *const *host_out,
                                 void *const *dev_in, void *const *dev_out, int nsteps, void *stream) {
    if (!p) return fail(nullptr, STENCIL_EINVAL, "plan is NULL");
    if (!host_in || !host_out) return fail(p, STENCIL_EINVAL, "host_in / host_out is NULL");
    for (int q = 0; q < p->nfields; ++q)
        if (!host_in[q] || !host_out[q])
            return fail(p, STENCIL_EINVAL, "host field " + std::to_string(q) + " is NULL");
    stencil_status st = check_device(p);
    if (st != STENCIL_OK) return st;
    if ((st = check_ptrs(p, dev_in, "dev_in")) != STENCIL_OK) return st;
    if ((st = check_ptrs(p, dev_out, "dev_out")) != STENCIL_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    for (int q = 0; q < p->nfields; ++q)
        CK(p, cudaMemcpyAsync(dev_in[q], host_in[q], p->bytes_per_field, cudaMemcpyHostToDevice, s), "copy in");
    if ((st = stencil_step(p, dev_in, dev_out, nsteps, stream)) != STENCIL_OK) return st;
    for (int q = 0; q < p->nfields; ++q)
        CK(p, cudaMemcpyAsync(host_out[q], dev_out[q], p->bytes_per_field, cudaMemcpyDeviceToHost, s), "copy out");
    return read_err(p, s);
}

stencil_status stencil_substep(stencil_t p, void *const *fin, void *const *fout, int substep, void *stream) {
    if (!p) return fail(nullptr, STENCIL_EINVAL, "plan is NULL");
    if (p->kind != STENCIL_MHD8) return fail(p, STENCIL_EINVAL, "stencil_substep needs an MHD8 plan");
    if (substep < 0 || substep > 2) return fail(p, STENCIL_EINVAL, "substep must be 0, 1 or 2");
    stencil_status st = check_device(p);
    if (st != STENCIL_OK) return st;
    if ((st = check_ptrs(p, fin, "fields_in")) != STENCIL_OK) return st;
    if ((st = check_ptrs(p, fout, "fields_out")) != STENCIL_OK) return st;
    for (int q = 0; q < 8; ++q)
        for (int r = 0; r < 8; ++r)
            if (fin[q] == fout[r]) return fail(p, STENCIL_EINVAL, "fields_in and fields_out alias");
    cudaStream_t s = (cudaStream_t)stream;
    CK(p, launch_halo_fill(p->geom, p->radius, p->esize, ptrs(fin, 8), 8, s, p->bc == STENCIL_BC_PERIODIC),
       "halo_fill launch");
    if (substep == 0 && p->storage != STENCIL_F64) {
        const size_t ncell = (size_t)(p->geom.n[0] * p->geom.n[1] * p->geom.n[2]);
        CK(p, cudaMemsetAsync(p->kc[0], 0, 8 * ncell * p->esize, s), "clear Kahan terms");
    }
    return run_pass(p, fin, fout, 1, substep, s);
}

stencil_status stencil_mhd_rhs(stencil_t p, void *const *fields, void *const *rhs, void *stream) {
    if (!p) return fail(nullptr, STENCIL_EINVAL, "plan is NULL");
    if (p->kind != STENCIL_MHD8) return fail(p, STENCIL_EINVAL, "stencil_mhd_rhs needs an MHD8 plan");
    stencil_status st = check_device(p);
    if (st != STENCIL_OK) return st;
    if ((st = check_ptrs(p, fields, "fields")) != STENCIL_OK) return st;
    if ((st = check_ptrs(p, rhs, "rhs")) != STENCIL_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    CK(p, launch_halo_fill(p->geom, p->radius, p->esize, ptrs(fields, 8), 8, s, p->bc == STENCIL_BC_PERIODIC),
       "halo_fill launch");
    int box[3];
    mhd_box(storage_code(p->storage), p->variant, box);
    MhdMaps maps;
    for (int q = 0; q < 8; ++q) {
        st = tma_map(p, fields[q], box, &maps.m[q]);
        if (st != STENCIL_OK) return st;
    }
    Ptrs8 none{};
    CK(p, launch_mhd(storage_code(p->storage), 1, 0, maps, none, nullptr, nullptr, ptrs(rhs, 8), p->geom, p->mconst,
                     false, p->err, s, p->variant, p->zmode),
       "mhd rhs launch");
    return STENCIL_OK;
}

static stencil_status read_err(stencil_t p, cudaStream_t s) {
    unsigned h = 0;
    CK(p, cudaMemcpyAsync(&h, p->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "read error word");
    CK(p, cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (h) {
        CK(p, cudaMemsetAsync(p->err, 0, sizeof(unsigned), s), "clear error word");
        CK(p, cudaStreamSynchronize(s), "cudaStreamSynchronize");
        if (h & ERR_TIMEOUT) return fail(p, STENCIL_ETIMEOUT, "a bounded mbarrier wait expired in a stencil kernel");
    }
    return STENCIL_OK;
}

stencil_status stencil_selftest_wait(stencil_t p, int64_t limit_ns, void *stream) {
    if (!p) return fail(nullptr, STENCIL_EINVAL, "plan is NULL");
    stencil_status st = check_device(p);
    if (st != STENCIL_OK) return st;
    const uint64_t lim = (uint64_t)std::min<int64_t>(std::max<int64_t>(limit_ns, 1000), 2000000000);
    CK(p, launch_selftest_wait(lim, p->err, (cudaStream_t)stream), "self-test launch");
    return STENCIL_OK;
}

stencil_status stencil_sync(stencil_t p, void *stream) {
    if (!p) return fail(nullptr, STENCIL_EINVAL, "plan is NULL");
    stencil_status st = check_device(p);
    if (st != STENCIL_OK) return st;
    return read_err(p, (cudaStream_t)stream);
}

stencil_status stencil_field_norms(stencil_t p, void *const *fields, double *out, void *stream) {
    if (!p) return fail(nullptr, STENCIL_EINVAL, "plan is NULL");
    if (!out) return fail(p, STENCIL_EINVAL, "out is NULL");
    stencil_status st = check_device(p);
    if (st != STENCIL_OK) return st;
    if ((st = check_ptrs(p, fields, "fields")) != STENCIL_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const bool mass = p->kind == STENCIL_MHD8;
    CK(p, launch_norms(storage_code(p->storage), ptrs(fields, p->nfields), p->nfields, p->geom, mass, p->partials,
                       p->red_out, s),
       "norms launch");
    std::vector<double> buf(p->nfields * 4);
    CK(p, cudaMemcpyAsync(buf.data(), p->red_out, sizeof(double) * buf.size(), cudaMemcpyDeviceToHost, s),
       "copy norms");
    st = read_err(p, s);
    if (st != STENCIL_OK) return st;
    for (int q = 0; q < p->nfields; ++q)
        for (int c = 0; c < 3; ++c) out[3 * q + c] = buf[4 * q + c];
    if (mass) out[3 * p->nfields] = buf[3] * p->par.dx[0] * p->par.dx[1] * p->par.dx[2];
    return STENCIL_OK;
}

static int num_variants(stencil_t p) {
    if (p->kind == STENCIL_DIFFUSION && p->ndim == 2) return p->storage == STENCIL_F32 ? 3 : 1;
    if (p->kind == STENCIL_DIFFUSION)
        return p->ndim == 3 ? diffusion_num_variants(storage_code(p->storage), p->radius) : 1;
    if (p->kind == STENCIL_MHD8) return mhd_num_variants(storage_code(p->storage));
    return 1;
}

static const char *variant_name(stencil_t p, int v) {
    if (p->kind == STENCIL_MAXFILTER) return "doubling_chunk4096";
    if (p->kind == STENCIL_XCORR && !xcorr_blocked(p)) return "wide_register_blocked";
    // FP64 sweeps one output per thread over a runtime chunk length; the other types use
    // 2184-cell chunks and 9-output register windows
    const bool f64 = p->storage == STENCIL_F64;
    if (p->kind == STENCIL_DIFFUSION && p->ndim == 1)
        return f64 ? "xcorr_folded_runtime_chunk_scalar_temporal_blocking" : "xcorr_folded_chunk2184_v9_temporal_blocking";
    if (p->kind == STENCIL_DIFFUSION && p->ndim == 2)
        return v == 1 ? "stream2d_tb2" : v == 2 ? "stream2d_tb4" : "tile2d_32vx_by8_ry4";
    if (p->kind == STENCIL_DIFFUSION) return diffusion_variant_name(storage_code(p->storage), p->radius, v);
    if (p->kind == STENCIL_MHD8) return mhd_variant_name(storage_code(p->storage), v);
    return f64 ? "runtime_chunk_scalar_temporal_blocking" : "chunk2184_v9_temporal_blocking";
}

stencil_status stencil_get_variant(stencil_t p, int *variant, int *count, const char **name) {
    if (!p) return fail(nullptr, STENCIL_EINVAL, "plan is NULL");
    if (variant) *variant = p->variant;
    if (count) *count = num_variants(p);
    if (name) *name = variant_name(p, p->variant);
    return STENCIL_OK;
}

stencil_status stencil_set_variant(stencil_t p, int variant) {
    if (!p) return fail(nullptr, STENCIL_EINVAL, "plan is NULL");
    if (variant < 0 || variant >= num_variants(p))
        return fail(p, STENCIL_EINVAL, "variant out of range");
    p->variant = variant;
    return STENCIL_OK;
}

// Streaming 3D kernels have a z-chunk length to tune besides the tile shape.
static int num_zmodes(stencil_t p) {
    return ((p->kind == STENCIL_DIFFUSION && p->ndim == 3) || p->kind == STENCIL_MHD8) ? ZMODES : 1;
}

stencil_status stencil_autotune(stencil_t p, void *const *fin, void *const *fout, int nsteps, int reps,
                                void *stream) {
    if (!p) return fail(nullptr, STENCIL_EINVAL, "plan is NULL");
    if (nsteps < 1 || reps < 1) return fail(p, STENCIL_EINVAL, "nsteps and reps must be >= 1");
    const std::string key = tune_key(p, nsteps);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        tune_load_locked(tune_path());
        auto it = g_tune.find(key);
        if (it != g_tune.end())
            for (int v = 0; v < num_variants(p); ++v)
                if (it->second.variant == variant_name(p, v) && it->second.zmode < num_zmodes(p)) {
                    p->variant = v;
                    p->zmode = it->second.zmode;
                    p->tuned_from_cache = 1;
                    p->tuned_ms = it->second.ms;
                    return STENCIL_OK;
                }
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    CK(p, cudaEventCreate(&e0), "cudaEventCreate");
    CK(p, cudaEventCreate(&e1), "cudaEventCreate");
    const int keep_v = p->variant, keep_z = p->zmode;
    int best = -1, best_z = 0;
    float best_ms = 0.f;
    for (int v = 0; v < num_variants(p); ++v)
        for (int z = 0; z < num_zmodes(p); ++z) {
            p->variant = v;
            p->zmode = z;
            if (stencil_step(p, fin, fout, nsteps, stream) != STENCIL_OK) continue;  // failed launch: discard
            if (cudaEventRecord(e0, s) != cudaSuccess) break;
            bool ok = true;
            for (int r = 0; r < reps && ok; ++r) ok = stencil_step(p, fin, fout, nsteps, stream) == STENCIL_OK;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ok && read_err(p, s) == STENCIL_OK && (best < 0 || ms < best_ms)) {
                best = v;
                best_z = z;
                best_ms = ms;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best < 0) {
        p->variant = keep_v;
        p->zmode = keep_z;
        return fail(p, STENCIL_ECUDA, "no kernel variant launched successfully");
    }
    p->variant = best;
    p->zmode = best_z;
    p->tuned_from_cache = 0;
    p->tuned_ms = best_ms / reps;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        const TuneRec rec{variant_name(p, best), best_z, p->tuned_ms};
        tune_put_locked(key, rec);
        const std::string path = tune_path();
        if (!path.empty()) {
            std::ofstream out(path, std::ios::app);
            if (out) out << key << '\t' << rec.variant << '\t' << rec.zmode << '\t' << rec.ms << '\n';
        }
    }
    return STENCIL_OK;
}

stencil_status stencil_set_zmode(stencil_t p, int zmode) {
    if (!p) return fail(nullptr, STENCIL_EINVAL, "plan is NULL");
    if (zmode < 0 || zmode >= num_zmodes(p)) return fail(p, STENCIL_EINVAL, "z-chunk mode out of range for this plan");
    p->zmode = zmode;
    return STENCIL_OK;
}

stencil_status stencil_autotune_status(stencil_t p, int *from_cache, int *zmode, float *ms) {
    if (!p) return fail(nullptr, STENCIL_EINVAL, "plan is NULL");
    if (from_cache) *from_cache = p->tuned_from_cache;
    if (zmode) *zmode = p->zmode;
    if (ms) *ms = p->tuned_ms;
    return STENCIL_OK;
}

stencil_status stencil_field_norms_noalloc(void *const *fields, int nfields, stencil_dtype storage,
                                           const int64_t dims[3], const int64_t padded[3],
                                           const int64_t origin[3], double mass_volume, double *out_dev,
                                           void *stream) {
    g_create_detail.clear();
    const int maxf = norms_static_max_fields();
    if (nfields < 1 || nfields > maxf)
        return fail(nullptr, STENCIL_EINVAL,
                    "nfields " + std::to_string(nfields) + " out of range 1.." + std::to_string(maxf) +
                        " (the allocation-free scratch holds at most " + std::to_string(maxf) + " fields)");
    if ((int)storage < 0 || (int)storage > 3) return fail(nullptr, STENCIL_EINVAL, "unknown dtype");
    if (!fields || !dims || !padded || !origin || !out_dev)
        return fail(nullptr, STENCIL_EINVAL, "a pointer argument is NULL");
    // element-aligned fields and an 8-byte aligned result: a misaligned address would fault
    // in the kernels
    const int es = esize_of(storage);
    for (int q = 0; q < nfields; ++q) {
        if (!fields[q]) return fail(nullptr, STENCIL_EINVAL, "fields[" + std::to_string(q) + "] is NULL");
        if (reinterpret_cast<uintptr_t>(fields[q]) % es != 0)
            return fail(nullptr, STENCIL_EINVAL,
                        "fields[" + std::to_string(q) + "] is not aligned to its " + std::to_string(es) +
                            "-byte element size");
    }
    if (reinterpret_cast<uintptr_t>(out_dev) % sizeof(double) != 0)
        return fail(nullptr, STENCIL_EINVAL, "out_dev is not 8-byte aligned");
    Geom g{};
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 1 || origin[a] < 0 || padded[a] < origin[a] + dims[a])
            return fail(nullptr, STENCIL_EINVAL, "inconsistent dims / padded / origin on axis " + std::to_string(a));
        g.n[a] = dims[a];
        g.off[a] = origin[a];
        g.pad[a] = padded[a];
    }
    cudaError_t e = launch_norms_noalloc(storage_code(storage), ptrs(fields, nfields), nfields, g, mass_volume,
                                         out_dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "allocation-free norms launch");
    return STENCIL_OK;
}

}  // extern "C"
