// lbm_api.cu -- the C ABI declared in include/lbm.h: configuration checks,
// the handle and its device memory, AA parity bookkeeping, schedule dispatch
// and the checkpointed adjoint driver.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "d3q19.cuh"
#include "ksweep_api.h"
#include "lattice.cuh"
#include "lbm.h"
#include "ops.h"

using namespace lbm;

struct lbm_handle {
    lbm_config cfg;
    cudaStream_t stream;
    int device;
    const StorageOps *ops;
    HostGeom hg;
    int64_t nxp;
    bool force;
    bool owns;
    void *base;
    size_t bytes;
    void *f;       // populations
    void *f2;      // second lattice (TWO_LATTICE)
    bool m3;           // MERGED runs the shadow-shell sweep
    ShellInfo si;
    void *G3[2];       // shadow of the tile shells: current / next
    void *Z3;          // periodic z: per-tile values of the image planes
    void *ZC;          // z split into chunks: copy of the planes next to each chunk boundary
    int g3cur;
    bool g3fresh;      // G3[g3cur] mirrors the shell cells of f
    // cached CUDA graph of GRAPH_STEPS time steps from state gfrom to gto,
    // captured and replayed on an internal stream ordered after / before the
    // handle's stream with an event (the legacy default stream cannot be
    // captured)
    cudaGraphExec_t gexec;
    cudaStream_t gstream;
    cudaEvent_t gev;
    // adjoint backward: segment recomputes run on astream, overlapping the
    // adjoint steps of the segment after them on the handle's stream
    cudaStream_t astream;
    cudaEvent_t aev[5];  // start, recompute done (per buffer), adjoint done (per buffer)
    struct StepState {
        int parity, g3cur;
        bool g3fresh;
        void *f, *f2;
        bool operator==(const StepState &o) const
        {
            return parity == o.parity && g3cur == o.g3cur && g3fresh == o.g3fresh && f == o.f && f2 == o.f2;
        }
    } gfrom, gto;
    CUtensorMap tmap;  // TMA descriptor of f (MERGED)
    CUtensorMap tmapz; // the same over ZC (shadow-shell sweep with si.nzc > 1)
    bool ns;           // MERGED runs the neighbour-synchronised sweep
    int *prog;         // its progress words, one per tile
    CUtensorMap tmapns;  // its copy box: tile + halo, all 19 directions
    int *status;       // device status word: a bit per sweep whose bounded wait gave up
    double *partial;
    double *red_out;
    int *flag;
    int red_blocks;
    int parity;
    int64_t t;
    bool force_set;
    // per-kernel timing
    bool prof_on;
    std::vector<cudaEvent_t> *ev_pool;  // all events ever created
    std::vector<int> *rec_kind;         // kernel class of record k (events 2k, 2k+1)
    // adjoint driver state
    bool adj_ready;
    int64_t adj_T, adj_K;
    void *adj_work;
    size_t adj_bytes;
};

static void drop_graph(lbm_handle *h)
{
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
}

static void free_graph_stream(lbm_handle *h)
{
    drop_graph(h);
    if (h->gev) cudaEventDestroy(h->gev);
    if (h->gstream) cudaStreamDestroy(h->gstream);
    h->gev = nullptr;
    h->gstream = nullptr;
    for (cudaEvent_t &e : h->aev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    if (h->astream) cudaStreamDestroy(h->astream);
    h->astream = nullptr;
}

namespace {

constexpr size_t ALIGN = 256;
inline size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

const StorageOps *ops_for(int storage)
{
    switch (storage) {
    case LBM_STORAGE_F64: return &ops_f64();
    case LBM_STORAGE_F32: return &ops_f32();
    case LBM_STORAGE_F32S: return &ops_f32s();
    case LBM_STORAGE_F16S: return &ops_f16s();
    case LBM_STORAGE_BF16S: return &ops_bf16s();
    default: return nullptr;
    }
}

// Velocities of the configuration's lattice (lattice 0 is D3Q19).
inline int lat_q(const lbm_config &c) { return c.lattice == 0 ? 19 : c.lattice; }

// The launch table of a configuration: the D3Q19 kernels of its storage
// format, or the single-step D3Q15 / D3Q27 kernels.
const StorageOps *ops_for_cfg(const lbm_config &c)
{
    const int q = lat_q(c);
    if (q == 19) return ops_for(c.storage);
    switch (c.storage) {
    case LBM_STORAGE_F64: return ops_dq_f64(q);
    case LBM_STORAGE_F32: return ops_dq_f32(q);
    case LBM_STORAGE_F32S: return ops_dq_f32s(q);
    case LBM_STORAGE_F16S: return ops_dq_f16s(q);
    case LBM_STORAGE_BF16S: return ops_dq_bf16s(q);
    default: return nullptr;
    }
}

// Row pitch: nx rounded up to 16 elements.
inline int64_t pitch_of(const lbm_config &c) { return (c.nx + 15) / 16 * 16; }

inline int64_t state_elems(const lbm_config &c) { return (int64_t)lat_q(c) * c.nz * c.ny * pitch_of(c); }

size_t elem_size_of(int storage)
{
    switch (storage) {
    case LBM_STORAGE_F64: return 8;
    case LBM_STORAGE_F32:
    case LBM_STORAGE_F32S: return 4;
    default: return 2;
    }
}
size_t real_size_of(int storage) { return storage == LBM_STORAGE_F64 ? 8 : 4; }

// The shadow-shell sweep serves MERGED where the neighbour-synchronised
// one cannot run (and z has at least two planes when it is periodic); where
// neither can, MERGED runs the AA pair.
int sm_count();

// The neighbour-synchronised sweep serves MERGED when every face is a wall or lid, the format has the sweep, all tiles can be
// resident at once and they are at least half as many as the SMs (fewer
// tiles leave SMs idle; the shadow-shell sweep splits z for them).  The
// environment variable LBM_MERGED_SWEEP=shadow selects the shadow-shell
// sweep instead, LBM_MERGED_SWEEP=neighbour this one whenever it can run
// (any tile count up to the resident limit).
// The kernels' collision variant (COLL_*) of a configuration.
int coll_of(const lbm_config &c)
{
    switch (c.collision) {
    case LBM_COLLISION_TRT: return COLL_TRT;
    case LBM_COLLISION_REG: return COLL_REG;
    case LBM_COLLISION_MRT: return COLL_MRT;
    default: return COLL_BGK;
    }
}

bool uses_ns(const lbm_config &c, const ShellInfo &si)
{
    if (c.variant != LBM_VARIANT_MERGED || lat_q(c) != 19) return false;
    bool any_count = false;
    if (const char *e = getenv("LBM_MERGED_SWEEP")) {
        if (strcmp(e, "shadow") == 0) return false;
        any_count = strcmp(e, "neighbour") == 0;
    }
    for (int k = 0; k < 6; ++k)
        if (c.face_bc[k] == LBM_BC_PERIODIC) return false;
    const StorageOps *o = ops_for(c.storage);
    if (!o->nsweep || o->ns_ty != o->m3_ty) return false;
    const int64_t tiles = (int64_t)si.ntx * si.nty, sms = sm_count();
    const int per = o->nsweep_ctas_per_sm(c.force_mode != LBM_FORCE_NONE, coll_of(c));
    return per > 0 && tiles <= (int64_t)per * sms && (any_count || 2 * tiles >= sms);
}

// si: the tiles of c (shell_info), computed once per query or creation.
bool uses_m3(const lbm_config &c, const ShellInfo &si)
{
    if (c.variant != LBM_VARIANT_MERGED || lat_q(c) != 19) return false;
    if (uses_ns(c, si)) return false;
    // the shadow-shell sweep is built for BGK only
    if (c.collision != LBM_COLLISION_BGK) return false;
    if (c.face_bc[4] == LBM_BC_PERIODIC && c.nz < 2) return false;
    // the sweep indexes one shadow copy with 32-bit offsets
    return (double)si.gplane * (double)c.nz < 2147483647.0;
}

// Streaming multiprocessors of the current device (152 when it cannot be
// queried, e.g. on a host without a GPU sizing a buffer).
int sm_count()
{
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
        return v;
    cudaGetLastError();
    return 152;
}

ShellInfo shell_info(const lbm_config &c)
{
    ShellInfo si;
    memset(&si, 0, sizeof(si));
    const StorageOps *o = ops_for(c.storage);
    si.ntx = (int)((c.nx + 31) / 32);
    si.nty = (int)((c.ny + o->m3_ty - 1) / o->m3_ty);
    si.hb = (int)(c.ny / si.nty);
    si.rem = (int)(c.ny % si.nty);
    si.gplane = (int64_t)si.ntx * si.nty * Q * o->m3_nsp;
    // z chunks of at least 4 planes, one CTA per tile and chunk (not with
    // periodic z, whose march wraps): the count that minimises waves of CTAs
    // (one per SM) x planes per CTA, a chunk costing about 3 planes more
    // than its own (the march prologue and the even steps of the planes
    // next to it); kept at 1 unless that saves 5% or more
    si.nzc = 1;
    si.mute = -1;
    if (c.face_bc[4] != LBM_BC_PERIODIC) {
        const int64_t tiles = (int64_t)si.ntx * si.nty, sms = sm_count();
        auto cost = [&](int64_t n) {
            return (double)((tiles * n + sms - 1) / sms) * ((double)c.nz / (double)n + (n > 1 ? 3.0 : 0.0));
        };
        double best = cost(1);
        const double one = best;
        for (int64_t n = 2; n <= c.nz / 4; ++n) {
            if (cost(n) < best) {
                best = cost(n);
                si.nzc = (int)n;
            }
        }
        if (best > 0.95 * one) si.nzc = 1;
        // explicit count (tuning): LBM_MERGED_ZCHUNKS, clamped to 1 .. nz / 4
        if (const char *env = getenv("LBM_MERGED_ZCHUNKS")) {
            const int64_t v = atoll(env), cap = c.nz / 4 > 1 ? c.nz / 4 : 1;
            if (v >= 1) si.nzc = (int)(v < cap ? v : cap);
        }
    }
    return si;
}

// Elements of the chunk-boundary copy: 19 x 2 (nzc - 1) planes.
int64_t zcopy_elems(const lbm_config &c, const ShellInfo &si)
{
    if (!uses_m3(c, si)) return 0;
    return si.nzc > 1 ? (int64_t)Q * 2 * (si.nzc - 1) * c.ny * pitch_of(c) : 0;
}

struct Layout {
    size_t f, f2, G3, Z3, ZC, prog, partial, red_out, flag, status, total;
};

Layout layout_of(const lbm_config &c, const ShellInfo &si)
{
    Layout L;
    const size_t es = elem_size_of(c.storage);
    const size_t pop = align_up((size_t)state_elems(c) * es);
    size_t off = 0;
    L.f = off; off += pop;
    L.f2 = off; if (c.variant == LBM_VARIANT_TWO_LATTICE || c.variant == LBM_VARIANT_KSTEP) off += pop;
    L.G3 = off;
    if (uses_m3(c, si)) off += 2 * align_up((size_t)(si.gplane * c.nz) * es);
    L.Z3 = off;
    if (uses_m3(c, si) && c.face_bc[4] == LBM_BC_PERIODIC) {
        off += align_up((size_t)si.ntx * si.nty * ops_for(c.storage)->m3_zsave * real_size_of(c.storage));
    }
    L.ZC = off; off += align_up((size_t)zcopy_elems(c, si) * es);
    L.prog = off;
    if (uses_ns(c, si)) off += align_up(sizeof(int) * NS_PROG_INTS * (size_t)si.ntx * si.nty);
    L.partial = off; off += align_up(sizeof(double) * 5 * RED_BLOCKS_MAX);
    L.red_out = off; off += align_up(sizeof(double) * 5);
    L.flag = off; off += align_up(sizeof(int));
    L.status = off; off += align_up(sizeof(int));
    L.total = off;
    return L;
}

HostGeom host_geom(const lbm_config &c)
{
    HostGeom h;
    memset(&h, 0, sizeof(h));
    h.nx = (int)c.nx; h.ny = (int)c.ny; h.nz = (int)c.nz;
    for (int a = 0; a < 3; ++a) h.per[a] = c.face_bc[2 * a] == LBM_BC_PERIODIC;
    for (int k = 0; k < 6; ++k) h.lid[k] = c.face_bc[k] == LBM_BC_LID;
    h.omega = 1.0 / c.tau;
    h.kf = 1.0 - 0.5 * h.omega;
    h.coll = coll_of(c);
    h.omega_m = h.coll == COLL_TRT ? 1.0 / (0.5 + c.trt_lambda / (c.tau - 0.5)) : h.omega;
    h.kf_m = 1.0 - 0.5 * h.omega_m;
    h.mrt_s3 = c.mrt_s3;
    h.mrt_s4 = c.mrt_s4;
    h.q = lat_q(c);
    auto lid_terms = [&](auto cxf, auto cyf, auto czf, auto wf) {
        for (int k = 0; k < h.q; ++k) {
            const double cu = cxf(k) * c.u_lid[0] + cyf(k) * c.u_lid[1] + czf(k) * c.u_lid[2];
            h.L[k] = 6.0 * wf(k) * c.rho_wall * cu;
        }
    };
    if (h.q == 15) lid_terms(DQ<15>::cx, DQ<15>::cy, DQ<15>::cz, DQ<15>::wgt);
    else if (h.q == 27) lid_terms(DQ<27>::cx, DQ<27>::cy, DQ<27>::cz, DQ<27>::wgt);
    else lid_terms(cx, cy, cz, wgt);
    if (c.force_mode == LBM_FORCE_UNIFORM)
        for (int a = 0; a < 3; ++a) h.Fu[a] = c.force_uniform[a];
    h.Ff = nullptr;
    return h;
}

// Keeps the handle's device current for the duration of an API call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

#define CK(call)                                   \
    do {                                           \
        if ((call) != cudaSuccess) return LBM_ECUDA; \
    } while (0)

// cuTensorMapEncodeTiled through the runtime's driver entry point (no
// link-time dependency on libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 4D map over f[q][z][y][x] (x extent nx, row pitch nxp, nzext planes per
// direction: nz for the lattice) with a box of one tile plane (tx x ty) and
// bq directions.
bool make_tmap(const lbm_config &c, int tx, int ty, int bq, void *f, CUtensorMap *map, int64_t nzext = 0)
{
    if (nzext <= 0) nzext = c.nz;
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    CUtensorMapDataType dt;
    switch (c.storage) {
    case LBM_STORAGE_F64: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT64; break;
    case LBM_STORAGE_F16S: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
    case LBM_STORAGE_BF16S: dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
    default: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
    }
    const cuuint64_t es = elem_size_of(c.storage), nxp = (cuuint64_t)pitch_of(c);
    const cuuint64_t dims[4] = {(cuuint64_t)c.nx, (cuuint64_t)c.ny, (cuuint64_t)nzext, (cuuint64_t)Q};
    const cuuint64_t strides[3] = {nxp * es, nxp * (cuuint64_t)c.ny * es, nxp * (cuuint64_t)c.ny * (cuuint64_t)nzext * es};
    const cuuint32_t box[4] = {(cuuint32_t)tx, (cuuint32_t)ty, 1u, (cuuint32_t)bq};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    return fn(map, dt, 4, f, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int check_dtype(int32_t dtype) { return dtype == LBM_DTYPE_F32 || dtype == LBM_DTYPE_F64 ? LBM_OK : LBM_EINVAL; }

const StorageOps *ops_for_dtype(int32_t dtype) { return dtype == LBM_DTYPE_F64 ? &ops_f64() : &ops_f32(); }


}  // namespace

// Bracket one launch with profiling events when profiling is on.
template <class F>
static cudaError_t timed(lbm_handle *h, int kind, F &&launch)
{
    if (!h->prof_on) return launch();
    const size_t k = h->rec_kind->size();
    while (h->ev_pool->size() < 2 * (k + 1)) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        h->ev_pool->push_back(e);
    }
    cudaError_t r = cudaEventRecord((*h->ev_pool)[2 * k], h->stream);
    if (r != cudaSuccess) return r;
    r = launch();
    if (r != cudaSuccess) return r;
    r = cudaEventRecord((*h->ev_pool)[2 * k + 1], h->stream);
    if (r != cudaSuccess) return r;
    h->rec_kind->push_back(kind);
    return cudaSuccess;
}

extern "C" {

void lbm_config_default(lbm_config *cfg)
{
    if (!cfg) return;
    memset(cfg, 0, sizeof(*cfg));
    cfg->nx = cfg->ny = cfg->nz = 32;
    cfg->tau = 0.6;
    for (int k = 0; k < 6; ++k) cfg->face_bc[k] = LBM_BC_PERIODIC;
    cfg->rho_wall = 1.0;
    cfg->storage = LBM_STORAGE_F32;
    cfg->variant = LBM_VARIANT_AA;
    cfg->force_mode = LBM_FORCE_NONE;
    cfg->collision = LBM_COLLISION_BGK;
    cfg->trt_lambda = 3.0 / 16.0;
    cfg->mrt_s3 = 1.0;
    cfg->mrt_s4 = 1.0;
    cfg->lattice = LBM_LATTICE_D3Q19;
}

int lbm_validate(const lbm_config *c)
{
    if (!c) return LBM_EINVAL;
    if (c->nx < 1 || c->ny < 1 || c->nz < 1) return LBM_EINVAL;
    if (c->ny > 65535 || c->nz > 65535 || c->nx > (1LL << 30)) return LBM_EINVAL;
    if ((double)c->nx * (double)c->ny * (double)c->nz > 2147483647.0) return LBM_EINVAL;
    if (!(c->tau > 0.5) || !isfinite(c->tau)) return LBM_EINVAL;
    for (int k = 0; k < 6; ++k)
        if (c->face_bc[k] < LBM_BC_PERIODIC || c->face_bc[k] > LBM_BC_LID) return LBM_EINVAL;
    for (int a = 0; a < 3; ++a)
        if ((c->face_bc[2 * a] == LBM_BC_PERIODIC) != (c->face_bc[2 * a + 1] == LBM_BC_PERIODIC)) return LBM_EINVAL;
    const double ul = sqrt(c->u_lid[0] * c->u_lid[0] + c->u_lid[1] * c->u_lid[1] + c->u_lid[2] * c->u_lid[2]);
    if (!(ul < 0.3)) return LBM_EINVAL;
    if (!(c->rho_wall > 0.0) || !isfinite(c->rho_wall)) return LBM_EINVAL;
    if (c->storage < LBM_STORAGE_F64 || c->storage > LBM_STORAGE_BF16S) return LBM_EINVAL;
    if (c->variant < LBM_VARIANT_TWO_LATTICE || c->variant > LBM_VARIANT_KSTEP) return LBM_EINVAL;
    if ((double)((c->nx + 15) / 16 * 16) * (double)c->ny * (double)c->nz > 2147483647.0) return LBM_EINVAL;
    if (c->force_mode < LBM_FORCE_NONE || c->force_mode > LBM_FORCE_FIELD) return LBM_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!isfinite(c->force_uniform[a])) return LBM_EINVAL;
    if (c->collision < LBM_COLLISION_BGK || c->collision > LBM_COLLISION_MRT) return LBM_EINVAL;
    if (!(c->mrt_s3 > 0.0 && c->mrt_s3 < 2.0) || !(c->mrt_s4 > 0.0 && c->mrt_s4 < 2.0)) return LBM_EINVAL;
    if (!(c->trt_lambda > 0.0) || !isfinite(c->trt_lambda)) return LBM_EINVAL;
    if (c->lattice != 0 && c->lattice != LBM_LATTICE_D3Q15 && c->lattice != LBM_LATTICE_D3Q19 &&
        c->lattice != LBM_LATTICE_D3Q27)
        return LBM_EINVAL;
    if (lat_q(*c) != 19 && c->collision == LBM_COLLISION_MRT) return LBM_EUNSUPPORTED;
    if (c->sweep_steps != 0 && c->sweep_steps != 3 && c->sweep_steps != 4) return LBM_EINVAL;
    if (c->variant == LBM_VARIANT_KSTEP &&
        (c->storage == LBM_STORAGE_F64 || lat_q(*c) != 19 || c->collision != LBM_COLLISION_BGK))
        return LBM_EUNSUPPORTED;
    return LBM_OK;
}

int lbm_required_bytes(const lbm_config *cfg, size_t *bytes)
{
    const int v = lbm_validate(cfg);
    if (v != LBM_OK) return v;
    if (!bytes) return LBM_EINVAL;
    *bytes = layout_of(*cfg, shell_info(*cfg)).total;
    return LBM_OK;
}

static int create_impl(const lbm_config *cfg, void *stream, void *buf, size_t bytes, bool own, lbm_handle **out)
{
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    const int v = lbm_validate(cfg);
    if (v != LBM_OK) return v;
    // the merged sweep's tiles and z chunks (current device, environment):
    // read once, so that the layout and the handle agree
    const ShellInfo si = shell_info(*cfg);
    const Layout L = layout_of(*cfg, si);
    lbm_handle *h = new (std::nothrow) lbm_handle;
    if (!h) return LBM_ENOMEM;
    memset((void *)h, 0, sizeof(*h));
    h->cfg = *cfg;
    h->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return LBM_ECUDA; }
    h->ops = ops_for_cfg(*cfg);
    h->hg = host_geom(*cfg);
    h->nxp = pitch_of(*cfg);
    h->force = cfg->force_mode != LBM_FORCE_NONE;
    h->force_set = cfg->force_mode != LBM_FORCE_FIELD;
    h->ev_pool = new (std::nothrow) std::vector<cudaEvent_t>();
    h->rec_kind = new (std::nothrow) std::vector<int>();
    if (!h->ev_pool || !h->rec_kind) {
        delete h->ev_pool;
        delete h->rec_kind;
        delete h;
        return LBM_ENOMEM;
    }
    if (own) {
        // stream-ordered allocation on the creation stream
        if (cudaMallocAsync(&buf, L.total, (cudaStream_t)stream) != cudaSuccess) {
            cudaGetLastError();
            delete h->ev_pool; delete h->rec_kind; delete h;
            return LBM_ENOMEM;
        }
        bytes = L.total;
    } else {
        if (!buf || ((uintptr_t)buf % ALIGN) != 0) { delete h->ev_pool; delete h->rec_kind; delete h; return LBM_EINVAL; }
        if (bytes < L.total) { delete h->ev_pool; delete h->rec_kind; delete h; return LBM_ENOMEM; }
    }
    h->owns = own;
    h->base = buf;
    h->bytes = bytes;
    char *b = (char *)buf;
    h->f = b + L.f;
    h->f2 = cfg->variant == LBM_VARIANT_TWO_LATTICE || cfg->variant == LBM_VARIANT_KSTEP ? b + L.f2 : nullptr;
    h->m3 = uses_m3(*cfg, si);
    h->ns = uses_ns(*cfg, si);
    if (h->ns) {
        h->si = si;
        h->prog = (int *)(b + L.prog);
    }
    if (h->m3) {
        h->si = si;
        const size_t gbytes = align_up((size_t)(h->si.gplane * cfg->nz) * elem_size_of(cfg->storage));
        h->G3[0] = b + L.G3;
        h->G3[1] = b + L.G3 + gbytes;
        h->Z3 = cfg->face_bc[4] == LBM_BC_PERIODIC ? b + L.Z3 : nullptr;
        h->ZC = h->si.nzc > 1 ? b + L.ZC : nullptr;
    }
    h->g3cur = 0;
    h->g3fresh = false;
    h->partial = (double *)(b + L.partial);
    h->red_out = (double *)(b + L.red_out);
    h->flag = (int *)(b + L.flag);
    h->status = (int *)(b + L.status);
    const int64_t n = cfg->nx * cfg->ny * cfg->nz;
    int64_t nb = (n + 255) / 256;
    h->red_blocks = (int)(nb < RED_BLOCKS_MAX ? nb : RED_BLOCKS_MAX);
    const bool tmap_ok = cfg->variant != LBM_VARIANT_MERGED ||
                         (h->ns ? make_tmap(*cfg, h->ops->ns_box_w, h->ops->ns_ty + 2, Q, h->f, &h->tmapns) :
                          h->m3 ? make_tmap(*cfg, 32, h->ops->m3_ty, 1, h->f, &h->tmap) &&
                                      (!h->ZC || make_tmap(*cfg, 32, h->ops->m3_ty, 1, h->ZC, &h->tmapz,
                                                           2 * (int64_t)(h->si.nzc - 1)))
                                : true);
    if (!tmap_ok ||
        cudaMemsetAsync(buf, 0, L.total, h->stream) != cudaSuccess) {
        if (own) cudaFreeAsync(buf, h->stream);
        delete h->ev_pool;
        delete h->rec_kind;
        delete h;
        return LBM_ECUDA;
    }
    *out = h;
    return LBM_OK;
}

int lbm_create(const lbm_config *cfg, void *stream, lbm_handle **out)
{
    return create_impl(cfg, stream, nullptr, 0, true, out);
}

int lbm_create_with_buffer(const lbm_config *cfg, void *stream, void *device_buffer, size_t bytes, lbm_handle **out)
{
    return create_impl(cfg, stream, device_buffer, bytes, false, out);
}

void lbm_destroy(lbm_handle *h)
{
    if (!h) return;
    {
        DeviceGuard g(h->device);
        cudaStreamSynchronize(h->stream);
        if (h->gstream) cudaStreamSynchronize(h->gstream);
        if (h->astream) cudaStreamSynchronize(h->astream);
        free_graph_stream(h);
        if (h->owns && h->base) {
            cudaFreeAsync(h->base, h->stream);
            cudaStreamSynchronize(h->stream);
        }
        if (h->ev_pool)
            for (cudaEvent_t e : *h->ev_pool) cudaEventDestroy(e);
    }
    delete h->ev_pool;
    delete h->rec_kind;
    delete h;
}

const char *lbm_strerror(int s)
{
    switch (s) {
    case LBM_OK: return "success";
    case LBM_EINVAL: return "invalid argument or configuration";
    case LBM_ENOMEM: return "device allocation failed or buffer too small";
    case LBM_ECUDA: return "CUDA runtime error";
    case LBM_ESTATE: return "call not valid in the current state";
    case LBM_ENONFINITE: return "non-finite value in the lattice";
    case LBM_ETIMEOUT: return "bounded device wait gave up";
    case LBM_EUNSUPPORTED: return "unsupported combination";
    default: return "unknown status";
    }
}

int lbm_lattice(int32_t *c, double *w)
{
    for (int i = 0; i < Q; ++i) {
        if (c) { c[3 * i] = cx(i); c[3 * i + 1] = cy(i); c[3 * i + 2] = cz(i); }
        if (w) w[i] = wgt(i);
    }
    return LBM_OK;
}

int lbm_lattice_q(int32_t q, int32_t *c, double *w)
{
    auto fill = [&](int n, auto cxf, auto cyf, auto czf, auto wf) {
        for (int i = 0; i < n; ++i) {
            if (c) { c[3 * i] = cxf(i); c[3 * i + 1] = cyf(i); c[3 * i + 2] = czf(i); }
            if (w) w[i] = wf(i);
        }
    };
    if (q == 0 || q == LBM_LATTICE_D3Q19) return lbm_lattice(c, w);
    if (q == LBM_LATTICE_D3Q15) fill(15, DQ<15>::cx, DQ<15>::cy, DQ<15>::cz, DQ<15>::wgt);
    else if (q == LBM_LATTICE_D3Q27) fill(27, DQ<27>::cx, DQ<27>::cy, DQ<27>::cz, DQ<27>::wgt);
    else return LBM_EINVAL;
    return LBM_OK;
}

int lbm_init_equilibrium(lbm_handle *h, const void *rho, const void *u, int32_t dtype)
{
    if (!h || check_dtype(dtype)) return LBM_EINVAL;
    DeviceGuard g(h->device);
    if (!g.ok) return LBM_ECUDA;
    CK(h->ops->init_eq(h->hg, h->nxp, h->f, rho, u, dtype, h->stream));
    h->parity = PARITY_NATURAL;
    h->g3fresh = false;
    h->t = 0;
    h->adj_ready = false;
    return LBM_OK;
}

int lbm_set_force(lbm_handle *h, const float *F)
{
    if (!h || !F) return LBM_EINVAL;
    if (h->cfg.force_mode != LBM_FORCE_FIELD) return LBM_ESTATE;
    h->hg.Ff = F;
    h->force_set = true;
    drop_graph(h);  // captured launches hold the old force pointer
    return LBM_OK;
}

// Enqueue n time steps with direct launches.
static int step_units(lbm_handle *h, int64_t n)
{
    const StorageOps &o = *h->ops;
    while (n > 0) {
        switch (h->cfg.variant) {
        case LBM_VARIANT_TWO_LATTICE: {
            CK(timed(h, LBM_KERNEL_TWO_LATTICE, [&] { return o.two_lattice(h->hg, h->nxp, h->force, h->f, h->f2, h->stream); }));
            void *t = h->f; h->f = h->f2; h->f2 = t;
            n -= 1; h->t += 1;
            break;
        }
        case LBM_VARIANT_KSTEP: {
            const int K = h->cfg.sweep_steps ? h->cfg.sweep_steps : 3;
            if (n >= K) {
                CK(timed(h, LBM_KERNEL_KSTEP, [&] {
                    return ksweep_launch(h->cfg.storage, h->hg, h->nxp, h->force, K, h->f, h->f2, h->stream);
                }));
                n -= K; h->t += K;
            } else {
                CK(timed(h, LBM_KERNEL_TWO_LATTICE, [&] { return o.two_lattice(h->hg, h->nxp, h->force, h->f, h->f2, h->stream); }));
                n -= 1; h->t += 1;
            }
            void *t = h->f; h->f = h->f2; h->f2 = t;
            break;
        }
        case LBM_VARIANT_AA:
            if (h->parity == PARITY_NATURAL) {
                CK(timed(h, LBM_KERNEL_AA_EVEN, [&] { return o.aa_even(h->hg, h->nxp, h->force, h->f, h->stream); }));
                h->parity = PARITY_A;
                h->g3fresh = false;
            } else {
                CK(timed(h, LBM_KERNEL_AA_ODD, [&] { return o.aa_odd(h->hg, h->nxp, h->force, h->f, h->stream); }));
                h->parity = PARITY_NATURAL;
                h->g3fresh = false;
            }
            n -= 1; h->t += 1;
            break;
        default:  // MERGED
            if (h->parity == PARITY_A) {
                CK(timed(h, LBM_KERNEL_AA_ODD, [&] { return o.aa_odd(h->hg, h->nxp, h->force, h->f, h->stream); }));
                h->parity = PARITY_NATURAL;
                h->g3fresh = false;
                n -= 1; h->t += 1;
            } else if (n >= 2 && h->ns) {
                CK(cudaMemsetAsync(h->prog, 0, sizeof(int) * NS_PROG_INTS * (size_t)h->si.ntx * h->si.nty, h->stream));
                CK(timed(h, LBM_KERNEL_MERGED, [&] {
                    return o.nsweep(h->hg, h->nxp, h->force, h->f, h->si, h->prog, &h->tmapns, h->status, h->stream);
                }));
                n -= 2; h->t += 2;
            } else if (n >= 2 && h->m3) {
                if (!h->g3fresh) {
                    CK(timed(h, LBM_KERNEL_SNAPSHOT, [&] {
                        return o.shell_gather(h->hg, h->nxp, h->f, h->G3[h->g3cur], h->si, h->stream);
                    }));
                    h->g3fresh = true;
                }
                if (h->ZC)
                    CK(timed(h, LBM_KERNEL_SNAPSHOT, [&] {
                        return o.zcopy(h->hg, h->nxp, h->f, h->ZC, h->si, h->stream);
                    }));
                CK(timed(h, LBM_KERNEL_MERGED, [&] {
                    return o.merged3(h->hg, h->nxp, h->force, h->f, h->G3[h->g3cur], h->G3[h->g3cur ^ 1], h->si,
                                     h->Z3, &h->tmap, &h->tmapz, h->status, h->stream);
                }));
                h->g3cur ^= 1;
                n -= 2; h->t += 2;
            } else {
                CK(timed(h, LBM_KERNEL_AA_EVEN, [&] { return o.aa_even(h->hg, h->nxp, h->force, h->f, h->stream); }));
                h->parity = PARITY_A;
                h->g3fresh = false;
                n -= 1; h->t += 1;
            }
            break;
        }
    }
    return LBM_OK;
}

static lbm_handle::StepState step_state(const lbm_handle *h)
{
    lbm_handle::StepState st;
    st.parity = h->parity;
    st.g3cur = h->g3cur;
    st.g3fresh = h->g3fresh;
    st.f = h->f;
    st.f2 = h->f2;
    return st;
}

static void set_step_state(lbm_handle *h, const lbm_handle::StepState &st)
{
    h->parity = st.parity;
    h->g3cur = st.g3cur;
    h->g3fresh = st.g3fresh;
    h->f = st.f;
    h->f2 = st.f2;
}

// Time steps per graph replay.  Long step(n) calls replay one captured
// block of launches instead of launching every kernel from the host.
constexpr int64_t GRAPH_STEPS = 32;

int lbm_step(lbm_handle *h, int64_t n)
{
    if (!h || n < 0) return LBM_EINVAL;
    if (!h->force_set) return LBM_ESTATE;
    DeviceGuard g(h->device);
    if (!g.ok) return LBM_ECUDA;
    if (n < GRAPH_STEPS || h->prof_on) return step_units(h, n);
    if (!h->gstream) {
        if (cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->gev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            free_graph_stream(h);
            return step_units(h, n);
        }
    }
    // the graph stream starts after everything already on the handle's stream
    CK(cudaEventRecord(h->gev, h->stream));
    CK(cudaStreamWaitEvent(h->gstream, h->gev, 0));
    cudaStream_t user = h->stream;
    int rc = LBM_OK;
    while (n >= GRAPH_STEPS) {
        const lbm_handle::StepState from = step_state(h);
        if (h->gexec && h->gfrom == from) {
            if (cudaGraphLaunch(h->gexec, h->gstream) != cudaSuccess) { rc = LBM_ECUDA; break; }
            set_step_state(h, h->gto);
            h->t += GRAPH_STEPS;
            n -= GRAPH_STEPS;
            continue;
        }
        // capture one block on the graph stream; on any failure fall back to
        // direct launches
        const int64_t t0 = h->t;
        if (cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            break;
        }
        h->stream = h->gstream;
        const int urc = step_units(h, GRAPH_STEPS);
        h->stream = user;
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(h->gstream, &graph);
        cudaGraphExec_t exec = nullptr;
        if (urc != LBM_OK || ec != cudaSuccess || !graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            set_step_state(h, from);
            h->t = t0;
            break;
        }
        cudaGraphDestroy(graph);
        const cudaError_t el = cudaGraphLaunch(exec, h->gstream);
        drop_graph(h);
        h->gexec = exec;
        h->gfrom = from;
        h->gto = step_state(h);
        if (el != cudaSuccess) { rc = LBM_ECUDA; break; }
        n -= GRAPH_STEPS;
    }
    // the handle's stream continues after the replays
    CK(cudaEventRecord(h->gev, h->gstream));
    CK(cudaStreamWaitEvent(h->stream, h->gev, 0));
    if (rc != LBM_OK) return rc;
    return step_units(h, n);
}

int lbm_time(const lbm_handle *h, int64_t *t)
{
    if (!h || !t) return LBM_EINVAL;
    *t = h->t;
    return LBM_OK;
}

int lbm_moments(lbm_handle *h, void *rho, void *u, int32_t dtype)
{
    if (!h || check_dtype(dtype)) return LBM_EINVAL;
    if (!h->force_set) return LBM_ESTATE;
    if (!rho && !u) return LBM_OK;
    DeviceGuard g(h->device);
    if (!g.ok) return LBM_ECUDA;
    CK(h->ops->moments(h->hg, h->nxp, h->force, h->parity, h->f, rho, u, dtype, h->stream));
    return LBM_OK;
}

int lbm_populations(lbm_handle *h, void *f_out, int32_t dtype)
{
    if (!h || !f_out || check_dtype(dtype)) return LBM_EINVAL;
    DeviceGuard g(h->device);
    if (!g.ok) return LBM_ECUDA;
    CK(h->ops->export_pop(h->hg, h->nxp, h->parity, h->f, f_out, dtype, h->stream));
    return LBM_OK;
}

int lbm_init_populations(lbm_handle *h, const void *f_in, int32_t dtype)
{
    if (!h || !f_in || check_dtype(dtype)) return LBM_EINVAL;
    DeviceGuard g(h->device);
    if (!g.ok) return LBM_ECUDA;
    CK(h->ops->import_pop(h->hg, h->nxp, h->f, f_in, dtype, h->stream));
    h->parity = PARITY_NATURAL;
    h->g3fresh = false;
    h->t = 0;
    h->adj_ready = false;
    return LBM_OK;
}

int lbm_reduce(lbm_handle *h, double *out)
{
    if (!h || !out) return LBM_EINVAL;
    if (!h->force_set) return LBM_ESTATE;
    DeviceGuard g(h->device);
    if (!g.ok) return LBM_ECUDA;
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
    CK(h->ops->reduce(h->hg, h->nxp, h->force, h->parity, h->f, h->partial, h->red_blocks, h->flag, h->red_out,
                      h->stream));
    int bad = 0, st = 0;
    CK(cudaMemcpyAsync(out, h->red_out, 5 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&bad, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (st) {
        CK(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
        return LBM_ETIMEOUT;
    }
    return bad ? LBM_ENONFINITE : LBM_OK;
}

int lbm_selftest_wait_timeout(lbm_handle *h)
{
    if (!h) return LBM_EINVAL;
    if (!h->ns || h->parity != PARITY_NATURAL || !h->force_set) return LBM_ESTATE;
    DeviceGuard g(h->device);
    if (!g.ok) return LBM_ECUDA;
    // one sweep in which the tile at the middle of the grid never publishes
    // its progress: its neighbours' waits for it run out, they give up, and
    // so does every tile waiting for them
    ShellInfo si = h->si;
    si.mute = (si.nty / 2) * si.ntx + si.ntx / 2;
    int st = 0;
    const bool ok =
        cudaMemsetAsync(h->status, 0, sizeof(int), h->stream) == cudaSuccess &&
        cudaMemsetAsync(h->prog, 0, sizeof(int) * NS_PROG_INTS * (size_t)si.ntx * si.nty, h->stream) == cudaSuccess &&
        h->ops->nsweep(h->hg, h->nxp, h->force, h->f, si, h->prog, &h->tmapns, h->status, h->stream) == cudaSuccess &&
        cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream) == cudaSuccess &&
        cudaMemsetAsync(h->status, 0, sizeof(int), h->stream) == cudaSuccess;
    if (!ok || cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_ECUDA;
    h->adj_ready = false;
    return st ? LBM_ETIMEOUT : LBM_OK;
}

int lbm_profile(lbm_handle *h, int32_t enable)
{
    if (!h) return LBM_EINVAL;
    if (enable) h->rec_kind->clear();
    h->prof_on = enable != 0;
    return LBM_OK;
}

int lbm_profile_read(lbm_handle *h, int32_t kernel, int64_t *launches, double *total_ms)
{
    if (!h || kernel < 0 || kernel >= LBM_KERNEL_COUNT) return LBM_EINVAL;
    DeviceGuard g(h->device);
    if (!g.ok) return LBM_ECUDA;
    int64_t cnt = 0;
    double ms = 0.0;
    for (size_t k = 0; k < h->rec_kind->size(); ++k) {
        if ((*h->rec_kind)[k] != kernel) continue;
        CK(cudaEventSynchronize((*h->ev_pool)[2 * k + 1]));
        float e = 0.f;
        CK(cudaEventElapsedTime(&e, (*h->ev_pool)[2 * k], (*h->ev_pool)[2 * k + 1]));
        ms += e;
        ++cnt;
    }
    if (launches) *launches = cnt;
    if (total_ms) *total_ms = ms;
    return LBM_OK;
}

// ---------------------------------------------------------------- adjoint

int lbm_adjoint_step(lbm_handle *h, const void *f_t, const void *lambda_in, void *lambda_out, int32_t dtype,
                     double *dLdF)
{
    if (h && (h->cfg.collision != LBM_COLLISION_BGK || lat_q(h->cfg) != 19)) return LBM_EUNSUPPORTED;
    if (!h || !f_t || !lambda_in || !lambda_out || lambda_in == lambda_out || check_dtype(dtype)) return LBM_EINVAL;
    if (!h->force_set) return LBM_ESTATE;
    DeviceGuard g(h->device);
    if (!g.ok) return LBM_ECUDA;
    CK(ops_for_dtype(dtype)->adjoint(h->hg, h->cfg.nx, h->force, f_t, lambda_in, lambda_out, dLdF, h->stream));
    return LBM_OK;
}

int lbm_adjoint_seed(lbm_handle *h, const void *dLdrho, const void *dLdu, void *lambda, int32_t dtype, double *dLdF)
{
    if (h && (h->cfg.collision != LBM_COLLISION_BGK || lat_q(h->cfg) != 19)) return LBM_EUNSUPPORTED;
    if (!h || !dLdu || !lambda || check_dtype(dtype)) return LBM_EINVAL;
    if (!h->force_set) return LBM_ESTATE;
    DeviceGuard g(h->device);
    if (!g.ok) return LBM_ECUDA;
    // the caller's lambda buffer first receives the canonical populations;
    // the seed kernel then replaces each cell's populations by its lambda
    CK(h->ops->export_pop(h->hg, h->nxp, h->parity, h->f, lambda, dtype, h->stream));
    CK(ops_for_dtype(dtype)->adjoint_seed(h->hg, h->cfg.nx, h->force, lambda, dLdrho, dLdu, dtype, lambda, dLdF,
                                          h->stream));
    return LBM_OK;
}

namespace {
// Workspace: the checkpoints f^0, f^K, f^2K, ... and f^T; two segment
// buffers, so that one segment is recomputed while the adjoint runs through
// the other, each with two states (the recompute's ping-pong) and the
// moments (rho, u) of the segment's K states, which is all of f^t the
// adjoint step reads; two adjoint buffers.  The forward pass steps through
// the two states of segment buffer 0.
struct AdjLayout {
    size_t state, lam, mom, ckpt0, nck, seg0, segb, lam0, total;
};
AdjLayout adj_layout(const lbm_handle *h, int64_t T, int64_t K)
{
    AdjLayout A;
    A.state = align_up((size_t)state_elems(h->cfg) * h->ops->elem_size);
    A.lam = align_up((size_t)state_elems(h->cfg) * h->ops->real_size);
    A.mom = align_up((size_t)(state_elems(h->cfg) / Q) * 4 * h->ops->real_size);
    A.nck = (size_t)((T + K - 1) / K) + 1;  // checkpoints at 0, K, 2K, ... plus f^T
    A.ckpt0 = 0;
    A.seg0 = A.nck * A.state;
    A.segb = 2 * A.state + (size_t)K * A.mom;  // one segment buffer
    A.lam0 = A.seg0 + 2 * A.segb;
    A.total = A.lam0 + 2 * A.lam;
    return A;
}
}  // namespace

int lbm_adjoint_workspace_bytes(const lbm_handle *h, int64_t T, int64_t K, size_t *bytes)
{
    if (!h || !bytes || T < 1 || K < 1) return LBM_EINVAL;
    if (lat_q(h->cfg) != 19) return LBM_EUNSUPPORTED;
    *bytes = adj_layout(h, T, K).total;
    return LBM_OK;
}

int lbm_adjoint_forward(lbm_handle *h, int64_t T, int64_t K, void *work, size_t work_bytes)
{
    if (h && (h->cfg.collision != LBM_COLLISION_BGK || lat_q(h->cfg) != 19)) return LBM_EUNSUPPORTED;
    if (!h || !work || T < 1 || K < 1 || ((uintptr_t)work % ALIGN) != 0) return LBM_EINVAL;
    if (!h->force_set) return LBM_ESTATE;
    const AdjLayout A = adj_layout(h, T, K);
    if (work_bytes < A.total) return LBM_ENOMEM;
    DeviceGuard g(h->device);
    if (!g.ok) return LBM_ECUDA;
    const StorageOps &o = *h->ops;
    char *w = (char *)work;
    const size_t sb = (size_t)state_elems(h->cfg) * o.elem_size;
    // f^0 in natural parity, exactly
    if (h->parity == PARITY_A) CK(o.raw_natural(h->hg, h->nxp, h->f, w + A.ckpt0, h->stream));
    else CK(cudaMemcpyAsync(w + A.ckpt0, h->f, sb, cudaMemcpyDeviceToDevice, h->stream));
    void *cur = w + A.seg0, *nxt = w + A.seg0 + A.state;
    CK(cudaMemcpyAsync(cur, w + A.ckpt0, sb, cudaMemcpyDeviceToDevice, h->stream));
    for (int64_t t = 0; t < T; ++t) {
        CK(o.two_lattice(h->hg, h->nxp, h->force, cur, nxt, h->stream));
        void *tmp = cur; cur = nxt; nxt = tmp;
        if ((t + 1) % K == 0 && t + 1 < T)
            CK(cudaMemcpyAsync(w + A.ckpt0 + (size_t)((t + 1) / K) * A.state, cur, sb, cudaMemcpyDeviceToDevice,
                               h->stream));
    }
    // f^T: kept for the seed and installed as the handle's state
    CK(cudaMemcpyAsync(w + (A.nck - 1) * A.state, cur, sb, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(h->f, cur, sb, cudaMemcpyDeviceToDevice, h->stream));
    h->parity = PARITY_NATURAL;
    h->g3fresh = false;
    h->t += T;
    h->adj_ready = true;
    h->adj_T = T;
    h->adj_K = K;
    h->adj_work = work;
    h->adj_bytes = work_bytes;
    return LBM_OK;
}

int lbm_adjoint_backward(lbm_handle *h, const void *dLdrho, const void *dLdu, int32_t dtype, void *dLdf0,
                         double *dLdF, void *work, size_t work_bytes)
{
    if (!h || !dLdu || check_dtype(dtype)) return LBM_EINVAL;
    if (!h->adj_ready || work != h->adj_work || work_bytes != h->adj_bytes) return LBM_ESTATE;
    DeviceGuard g(h->device);
    if (!g.ok) return LBM_ECUDA;
    const StorageOps &o = *h->ops;
    const int64_t T = h->adj_T, K = h->adj_K;
    const AdjLayout A = adj_layout(h, T, K);
    char *w = (char *)work;
    void *la = w + A.lam0, *lb = w + A.lam0 + A.lam;
    CK(o.adjoint_seed(h->hg, h->nxp, h->force, w + (A.nck - 1) * A.state, dLdrho, dLdu, dtype, la, dLdF, h->stream));
    if (!h->astream) {
        if (cudaStreamCreateWithFlags(&h->astream, cudaStreamNonBlocking) != cudaSuccess) return LBM_ECUDA;
        for (cudaEvent_t &e : h->aev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return LBM_ECUDA;
    }
    // Segments from the last to the first.  Segment s recomputes its states
    // from checkpoint s into buffer s % 2 on astream, keeping only their
    // moments, and its adjoint steps t1-1 .. t0 run from those on the
    // handle's stream once that is done.  The recompute of segment s-1 (the
    // other buffer) waits only for the adjoint of segment s+1, so it overlaps
    // the adjoint of segment s: the recompute streams at the HBM roofline
    // while the adjoint steps leave bandwidth unused.
    const int64_t nseg = (T + K - 1) / K;
    CK(cudaEventRecord(h->aev[0], h->stream));
    CK(cudaStreamWaitEvent(h->astream, h->aev[0], 0));
    for (int64_t s = nseg - 1; s >= 0; --s) {
        const int b = (int)(s & 1);
        const int64_t t0 = s * K, t1 = (t0 + K < T) ? t0 + K : T;
        char *base = w + A.seg0 + (size_t)b * A.segb;
        char *pp[2] = {base, base + A.state};
        auto mom = [&](int64_t t) -> void * { return base + 2 * A.state + (size_t)(t - t0) * A.mom; };
        if (s + 2 < nseg) CK(cudaStreamWaitEvent(h->astream, h->aev[3 + b], 0));
        const void *cur = w + A.ckpt0 + (size_t)s * A.state;
        for (int64_t t = t0; t + 1 < t1; ++t) {
            void *nxt = pp[(t - t0) & 1];
            CK(o.two_lattice_mom(h->hg, h->nxp, h->force, cur, nxt, mom(t), h->astream));
            cur = nxt;
        }
        CK(o.adj_moments(h->hg, h->nxp, h->force, cur, mom(t1 - 1), h->astream));
        CK(cudaEventRecord(h->aev[1 + b], h->astream));
        CK(cudaStreamWaitEvent(h->stream, h->aev[1 + b], 0));
        for (int64_t t = t1 - 1; t >= t0; --t) {
            CK(o.adjoint_mom(h->hg, h->nxp, h->force, mom(t), la, lb, dLdF, h->stream));
            void *tmp = la; la = lb; lb = tmp;
        }
        CK(cudaEventRecord(h->aev[3 + b], h->stream));
    }
    if (dLdf0) CK(o.pitched_to_canon(h->hg, h->nxp, la, dLdf0, dtype, Q, h->stream));
    return LBM_OK;
}

}  // extern "C"
