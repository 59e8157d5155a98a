/*
 * Host runtime of the GB300 Gaussian source-finder library: the C ABI of
 * include/sf.h, the per-context plan (taps, radii, inputs of the fused kernel,
 * launch shapes, shared-memory layout), run-time compilation of the kernels
 * for the exact radii of the filter bank, and the launches.
 *
 * Plan of sf_detect for a bank of filters (sigma_xy, sigma_z):
 *   1. x pass (Eq. 2 factor along x) once per distinct non-zero sigma_xy into
 *      a scratch cube the context owns; one launch handles up to four sigmas
 *      and reads the cube once;
 *   2. one fused launch, one CTA per statistics window: the inputs (the cube
 *      itself for sigma_xy = 0, the scratch cubes otherwise) are filtered
 *      along y and z for every filter, the window mean and standard deviation
 *      are formed (Sec. 3.3), and c > mean + k*std is OR-ed over all filters
 *      into the packed mask; a second pass over the window refilters only the
 *      x-planes whose maximum exceeds a threshold.
 * Windows whose shape the fused kernel cannot tile (wy % 8, wz % 32, thread
 * or shared-memory limits) run the composed path: per filter sf_filter into a
 * scratch cube, sf_stats, sf_threshold accumulating the mask.
 */
#include "sf.h"
#include "sf_kernel_abi.h"

#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <nvrtc.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <vector>

extern "C" const char *sf_embedded_kernel_source;   /* sf_kernels.cuh (generated) */
extern "C" const char *sf_embedded_abi_source;      /* sf_kernel_abi.h (generated) */

/* AOT kernels (sf_aot.cu) */
cudaError_t sf_launch_stats(const float *c, long long nx, long long ny, long long nz, int wx, int wy,
                            int wz, int nwx, int nwy, int nwz, float *mean, float *stdv, int fp64, int ddof,
                            cudaStream_t st);
size_t sf_local_yz_smem(int sy, int sz);
cudaError_t sf_launch_w_product(const float *d, const float *w, float *p, long long n, cudaStream_t st);
cudaError_t sf_launch_w_ratio(const float *num, const float *den, float *out, long long n, cudaStream_t st);
cudaError_t sf_launch_local_yz(const float *c, float *P, float *Q, long long nx, long long ny, long long nz, int sy,
                               int sz, cudaStream_t st);
bool sf_local_is_narrow(int sx, int sy, int sz);
cudaError_t sf_launch_local_direct(const float *c, long long nx, long long ny, long long nz, long long nw32,
                                   int sx, int sy, int sz, float k, float *mean, float *stdv, unsigned int *mask,
                                   int mode, int ddof, cudaStream_t st);
cudaError_t sf_launch_local_x(const float *c, const float *P, const float *Q, long long nx, long long ny,
                              long long nz, long long nw32, int sx, int sy, int sz, float k, float *mean,
                              float *stdv, unsigned int *mask, int mode, int ddof, cudaStream_t st);
cudaError_t sf_launch_threshold(const float *c, long long nx, long long ny, long long nz, int wx,
                                int wy, int wz, int nwy, int nwz, const float *mean,
                                const float *stdv, float k, unsigned int *mask, int accumulate,
                                cudaStream_t st);

namespace {

constexpr int kMaxRadius = 64;
constexpr int kMaxFilters = 64;
constexpr size_t kSmemLimit = 227 * 1024;

std::mutex g_err_mu;
std::string g_create_error;

/* ------------------------------------------------------------ taps ------ */
int radius_of(double sigma, double truncation)
{
    if (!(sigma > 0.0)) return 0;
    return (int)std::ceil(truncation * sigma);
}

/* Sampled Gaussian exp(-o^2 / 2 sigma^2), o = -R..R, scaled to unit sum. */
std::vector<double> gaussian_taps(double sigma, int R)
{
    std::vector<double> g(2 * R + 1, 1.0);
    if (R == 0) return g;
    double total = 0.0;
    for (int o = -R; o <= R; ++o) {
        g[o + R] = std::exp(-(double)o * o / (2.0 * sigma * sigma));
        total += g[o + R];
    }
    for (double &v : g) v /= total;
    return g;
}

struct Filt {
    float sxy = 0.f, sz = 0.f;
    int rxy = 0, rz = 0;
    std::vector<float> gxy, gz;   /* 2R+1 float taps */
    int slot = -1;                /* x-filtered scratch cube, -1 = none (sigma_xy == 0) */
};

struct DetectSource {
    int slot;                     /* -1 = the cube itself */
    int ry;
    std::vector<int> filters;     /* <= nzf entries */
    bool den = false;             /* Eq. 1 plans: the denominator of a (den, num) pair */
};

struct Launch {
    cudaKernel_t kernel = nullptr;
    dim3 grid, block;
    size_t smem = 0;
    int v = 1;   /* x passes: elements per lane */
};

/* ------------------------------------------------------------ JIT -------- */
std::mutex g_jit_mu;
std::map<std::string, cudaKernel_t> g_jit_cache;

/* tuning override from the environment (launch shapes only, never the math) */
int env_int(const char *name, int dflt)
{
    const char *v = std::getenv(name);
    return (v && *v) ? std::atoi(v) : dflt;
}

int device_cc(int dev, int *major, int *minor)
{
    if (cudaDeviceGetAttribute(major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) return -1;
    return 0;
}

sf_status jit_kernel(const std::string &prelude, const char *name, int dev, cudaKernel_t *out,
                     std::string &err)
{
    int major = 0, minor = 0;
    if (device_cc(dev, &major, &minor) != 0) {
        err = "cannot query the compute capability of the device";
        return SF_ECUDA;
    }
    const std::string arch = "--gpu-architecture=sm_" + std::to_string(major * 10 + minor) +
                             (major >= 9 ? "a" : "");
    std::string src = std::string(sf_embedded_abi_source) + "\n" + prelude + "\n" +
                      sf_embedded_kernel_source;
    const std::string key = arch + "\n" + name + "\n" + src;
    {
        std::lock_guard<std::mutex> lk(g_jit_mu);
        auto it = g_jit_cache.find(key);
        if (it != g_jit_cache.end()) {
            *out = it->second;
            return SF_OK;
        }
    }
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "sf_kernels.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        err = "nvrtcCreateProgram failed";
        return SF_EJIT;
    }
    /* diagnostics: SF_JIT_DUMP=<dir> writes each compiled source there (to
     * rebuild it offline), SF_JIT_VERBOSE=1 prints ptxas' resource usage */
    if (const char *dir = std::getenv("SF_JIT_DUMP")) {
        const std::string path = std::string(dir) + "/" + name + "_" +
                                 std::to_string(std::hash<std::string>{}(src)) + ".cu";
        if (FILE *fh = std::fopen(path.c_str(), "w")) {
            std::fwrite(src.data(), 1, src.size(), fh);
            std::fclose(fh);
        }
    }
    const bool verbose = env_int("SF_JIT_VERBOSE", 0) != 0;
    const char *opts[] = {arch.c_str(), "-std=c++17", "-lineinfo", "--fmad=true",
                          "-DSF_JIT=1", "--ptxas-options=-v"};
    const int nopt = (int)(sizeof(opts) / sizeof(opts[0])) - (verbose ? 0 : 1);
    nvrtcResult rc = nvrtcCompileProgram(prog, nopt, opts);
    if (verbose && rc == NVRTC_SUCCESS) {
        size_t n = 0;
        nvrtcGetProgramLogSize(prog, &n);
        std::string log(n, '\0');
        if (n) nvrtcGetProgramLog(prog, &log[0]);
        std::fprintf(stderr, "[sf jit] %s: %s\n", name, log.c_str());
    }
    if (rc != NVRTC_SUCCESS) {
        size_t n = 0;
        nvrtcGetProgramLogSize(prog, &n);
        std::string log(n, '\0');
        if (n) nvrtcGetProgramLog(prog, &log[0]);
        err = std::string("kernel compilation failed (") + nvrtcGetErrorString(rc) + "): " +
              log.substr(0, 4000);
        nvrtcDestroyProgram(&prog);
        return SF_EJIT;
    }
    size_t nbin = 0;
    nvrtcGetCUBINSize(prog, &nbin);
    std::vector<char> cubin(nbin);
    nvrtcGetCUBIN(prog, cubin.data());
    nvrtcDestroyProgram(&prog);
    cudaLibrary_t lib;
    cudaError_t ce = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (ce != cudaSuccess) {
        err = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(ce);
        return SF_ECUDA;
    }
    cudaKernel_t k;
    ce = cudaLibraryGetKernel(&k, lib, name);
    if (ce != cudaSuccess) {
        err = std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(ce);
        return SF_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_jit_mu);
    g_jit_cache.emplace(key, k);
    *out = k;
    return SF_OK;
}

const char *storage_ctype(int storage)
{
    return storage == SF_F16 ? "sf_f16" : storage == SF_BF16 ? "sf_bf16" : "float";
}

size_t storage_bytes(int storage) { return storage == SF_F32 ? 4 : 2; }

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

/* smallest stride >= need with (stride / 4) odd: conflict-free 16-byte rows */
int odd_quad_stride(int need)
{
    int s = (need + 3) / 4 * 4;
    if ((s / 4) % 2 == 0) s += 4;
    return s;
}

}  // namespace

/* ============================================================ context === */
struct sf_ctx {
    sf_config cfg{};
    std::vector<Filt> filt;
    int device = 0;
    long long nvox = 0, nw32 = 0;
    int nwx = 0, nwy = 0, nwz = 0, nwin = 0;
    size_t ebytes = 4;

    /* x pass */
    std::vector<float> xy_sigma;      /* distinct non-zero sigma_xy, slot order */
    std::vector<int> xy_radius;
    void *scratch = nullptr;          /* n_slots cubes, storage dtype */
    size_t cube_bytes = 0;
    int xv = 1;                       /* elements per lane */
    int xpf = 4;                      /* ring prefetch depth (register-ring form) */
    int xd = 0;                       /* shared-memory staging depth, 0 = register ring */
    int xthreads = 256;
    long long xseg = 0;
    std::vector<std::vector<int>> xgroups;   /* slots per x-pass launch */
    std::vector<Launch> xlaunch;
    /* rows that are not 16-byte multiples: the scratch slots have a padded z
     * stride zs, and the detect path's x pass (one element per lane) also
     * writes a padded copy of the cube into slot n_xy (the identity output),
     * so the window kernels read every input by TMA */
    long long zs = 0;
    bool dpad = false;                       /* the detect plan reads the padded layout */
    std::vector<std::vector<int>> xgroups_p; /* slots per padded x-pass launch (n_xy: the copy) */
    std::vector<Launch> xlaunch_p;

    /* fused detect */
    bool fused = false;
    std::vector<DetectSource> dsrc;
    int dnzf = 1, dP = 16, dthreads = 0, dHZ = 0, dCH = 0, dSROW = 0, dUROW = 0;
    int dRYM = 0, dRZM = 0;
    bool dtma = false;
    Launch dlaunch;
    std::vector<float> dtaps;
    std::vector<CUtensorMap> dmaps;   /* per input; the cube's is re-encoded per call */
    /* 16-bit storage: the window kernel with the spectral filters on the tensor cores */
    bool use_tc = false;
    Launch tclaunch;
    std::vector<unsigned char> tcb;   /* swizzled Toeplitz tap tiles (parameter block) */
    void *d_tct = nullptr;            /* the same tiles in device memory: the kernel's copy source */
    std::vector<CUtensorMap> tcmaps;  /* per input: swizzled A boxes (sigma_xy = 0) or slabs */
    int *err_flag = nullptr;          /* device flag set by kernels whose bounded wait expired */
    long long wait_ns = 2000000000LL; /* limit of the kernels' bounded waits */
    int stall_extra = 0;              /* test hook: x items each window waits for beyond its unit's */

    /* per-filter y/z filter kernels (sf_filter) and single-sigma x pass */
    std::map<int, Launch> flaunch;
    std::map<int, Launch> xsingle;    /* by slot */
    std::map<int, std::vector<float>> ftaps;
    float *filt_scratch = nullptr;    /* composed path: one filtered cube */
    float *stat_scratch = nullptr;    /* composed path: mean/std of one filter */

    /* host-buffer entry point (pipelined along x) */
    void *host_cube = nullptr;
    unsigned int *host_mask = nullptr;
    cudaStream_t hcopy[2] = {nullptr, nullptr}, hback = nullptr;
    cudaStream_t hcomp[2] = {nullptr, nullptr};   /* compute streams of the host pipeline */
    float *lscratch = nullptr;        /* local statistics: filtered cube, P, Q */
    float *wscratch = nullptr;        /* weighted form: product, numerator, denominator */
    float *wstats = nullptr;          /* weighted form: window mean / std of one filter */
    sf_ctx *boxtwin = nullptr;        /* the bank's radii with unit taps (printed Eq. 1 denominator) */
    sf_ctx *gausstwin = nullptr;      /* the same bank: its scratch holds the x-filtered weights */
    struct WPlan {                    /* fused Eq. 1 window kernel, per denominator reading */
        bool tried = false, ready = false, tma = false;
        Launch L;
        std::vector<float> taps;
        std::vector<DetectSource> srcs;
        std::vector<CUtensorMap> maps;
    } wplan[2];
    std::vector<cudaEvent_t> hev;

    /* stage timing: pairs of events per recorded stage instance */
    bool prof = false;
    struct Rec { int stage; cudaEvent_t a, b; int launches; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;

    /* persistent form: the cubes of a batched context (or the one cube of a
     * plain context when the autotuner prefers it), one launch per call */
    struct Cube {
        long long nx, ny, nz, nw32;
        int nwx, nwy, nwz, nwin;
        long long zs;                 /* z stride of the scratch cubes: nz, or nz padded to 16 bytes */
        size_t slot_bytes;            /* one x-filtered cube */
        void *slots;                  /* n_xy scratch cubes, and a copy of the cube where zs > nz */
        bool tma;
        bool pad;                     /* this plan reads the padded scratch (and the copy) by TMA */
        int xv;
    };
    bool batch = false;               /* created by sf_create_batch */
    /* sectioned form (Sec. 3.1: cubes larger than device memory): x sections
     * of sect_S planes plus sect_h halo planes on each side, each processed
     * by a context of the section's shape; sub[1] serves a last section that
     * ends in a partial statistics window */
    bool sectioned = false;
    long long sect_S = 0, sect_h = 0;
    sf_ctx *sub[2] = {nullptr, nullptr};
    long long sub_nx[2] = {0, 0};
    void *sbuf[2] = {nullptr, nullptr};             /* section inputs */
    unsigned int *smask[2] = {nullptr, nullptr};    /* section masks */
    bool use_persist = false;         /* sf_detect runs the persistent kernel */
    std::vector<Cube> cubes;
    void *bscratch = nullptr;         /* scratch of all cubes (batched contexts) */
    struct PersistPlan {
        int P = 8, minb = 3, pf = 2, xlanes = 1024, slab = 0;
        bool xbatch = false;   /* x pass as one batched launch before the windows */
    } pp;
    bool pready = false;
    Launch plaunch;
    std::vector<float> ptaps, pxtaps;
    int pnsrc = 0, psrow = 0, prym = 0;
    std::vector<DetectSource> psrc;
    std::vector<sf_unit> units;       /* static fields; pointers filled per call */
    std::vector<int> unit_cube;
    int n_items = 0;
    sf_unit *d_units = nullptr, *h_units = nullptr;
    sf_item *d_items = nullptr;
    CUtensorMap *d_maps = nullptr, *h_maps = nullptr;
    int *d_ctr = nullptr;             /* [0] head, [1 + u] x items done of unit u */
    sf_xcube *d_xcubes = nullptr, *h_xcubes = nullptr;   /* batched x pass table */
    Launch xblaunch;                  /* batched x pass */
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gstream = nullptr;
    cudaEvent_t gdone = nullptr;
    bool gpending = false;
    std::string tune_report;

    std::string err;
    bool dead = false;
};

namespace {

sf_status fail(sf_ctx *c, sf_status s, const char *fmt, ...)
{
    char buf[2048];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else {
        std::lock_guard<std::mutex> lk(g_err_mu);
        g_create_error = buf;
    }
    return s;
}

sf_status cuda_fail(sf_ctx *c, cudaError_t e, const char *what)
{
    if (c) c->dead = true;
    return fail(c, SF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

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
        if (ok && prev >= 0) cudaSetDevice(prev);
    }
};

sf_status launch(sf_ctx *c, const Launch &L, void **args, cudaStream_t st, const char *what)
{
    cudaLaunchConfig_t lc{};
    lc.gridDim = L.grid;
    lc.blockDim = L.block;
    lc.dynamicSmemBytes = L.smem;
    lc.stream = st;
    cudaError_t e = cudaLaunchKernelExC(&lc, (const void *)L.kernel, args);
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    return SF_OK;
}

sf_status set_smem(sf_ctx *c, cudaKernel_t k, size_t smem)
{
    cudaError_t e = cudaKernelSetAttributeForDevice(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)smem, c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaKernelSetAttributeForDevice");
    return SF_OK;
}

/* ---------------------------------------------------- x pass kernels --- */
/* x radius of a scratch slot; slot n_xy is the identity (the cube's copy) */
int slot_radius(const sf_ctx *c, int slot)
{
    return slot < (int)c->xy_radius.size() ? c->xy_radius[slot] : 0;
}

sf_status build_xpass(sf_ctx *c, const std::vector<int> &slots, Launch *L, int v = 0)
{
    if (v <= 0) v = c->xv;
    /* cp.async copies 4, 8 or 16 bytes: narrower lanes use the register ring */
    const int xd = v * (int)c->ebytes < 4 ? 0 : c->xd;
    const int nout = (int)slots.size();
    int r[4] = {0, 0, 0, 0}, rm = 0;
    for (int i = 0; i < nout; ++i) {
        r[i] = slot_radius(c, slots[i]);
        rm = std::max(rm, r[i]);
    }
    std::string p;
    p += "#define SF_KERNEL_XPASS 1\n";
    p += "#define SFX_NOUT " + std::to_string(nout) + "\n";
    for (int i = 0; i < 4; ++i) p += "#define SFX_R" + std::to_string(i) + " " + std::to_string(r[i]) + "\n";
    p += "#define SFX_RM " + std::to_string(rm) + "\n";
    p += "#define SFX_PF " + std::to_string(c->xpf) + "\n";
    p += "#define SFX_V " + std::to_string(v) + "\n";
    p += "#define SFX_THREADS " + std::to_string(c->xthreads) + "\n";
    p += "#define SFX_D " + std::to_string(xd) + "\n";
    p += std::string("typedef ") + storage_ctype(c->cfg.storage) + " sfx_t;\n";
    std::string err;
    sf_status s = jit_kernel(p, "sf_xpass", c->device, &L->kernel, err);
    if (s != SF_OK) return fail(c, s, "x pass: %s", err.c_str());
    const long long plane = c->cfg.ny * c->cfg.nz;
    const long long lanes = plane / v;
    const long long nseg = (c->cfg.nx + c->xseg - 1) / c->xseg;
    L->block = dim3(c->xthreads);
    L->grid = dim3((unsigned)((lanes + c->xthreads - 1) / c->xthreads), (unsigned)nseg);
    L->v = v;
    /* staged form: xd slots of one vector per thread */
    L->smem = xd > 0 ? (size_t)xd * c->xthreads * v * c->ebytes : 0;
    if (L->smem > 48 * 1024 && (s = set_smem(c, L->kernel, L->smem)) != SF_OK) return s;
    return SF_OK;
}

std::vector<float> xpass_taps(const sf_ctx *c, const std::vector<int> &slots)
{
    int rm = 0;
    for (int s : slots) rm = std::max(rm, slot_radius(c, s));
    std::vector<float> t(slots.size() * (rm + 1), 0.f);
    for (size_t i = 0; i < slots.size(); ++i) {
        if (slots[i] >= (int)c->xy_radius.size()) {
            t[i * (rm + 1)] = 1.f;   /* the identity: an exact copy */
            continue;
        }
        /* any filter of this slot carries its taps */
        for (const Filt &f : c->filt)
            if (f.slot == slots[i]) {
                for (int j = 0; j <= f.rxy; ++j) t[i * (rm + 1) + j] = f.gxy[f.rxy + j];
                break;
            }
    }
    return t;
}

sf_status run_xpass(sf_ctx *c, const Launch &L, const std::vector<int> &slots, const void *cube,
                    cudaStream_t st, long long x0 = 0, long long x1 = -1, bool padded = false)
{
    sf_xargs xa{};
    xa.src = cube;
    for (size_t i = 0; i < slots.size(); ++i)
        xa.dst[i] = (char *)c->scratch + (size_t)slots[i] * c->cube_bytes;
    xa.nx = c->cfg.nx;
    xa.plane = c->cfg.ny * c->cfg.nz;
    xa.lanes = xa.plane / L.v;
    xa.nz = c->cfg.nz;
    xa.ozs = padded ? c->zs : c->cfg.nz;
    xa.xseg = c->xseg;
    xa.xoff = 0;
    Launch LL = L;
    if (x1 >= 0) {
        /* one grid row over output planes [x0, x1) */
        xa.xoff = x0;
        xa.xseg = x1 - x0;
        LL.grid.y = 1;
    }
    std::vector<float> taps = xpass_taps(c, slots);
    void *args[] = {&xa, taps.data()};
    return launch(c, LL, args, st, "x pass launch");
}

/* ------------------------------------------- y/z kernels: shared bits --- */
struct YZShape {
    int WY, WZ, threads, HZ, CH, SROW, UROW, RYM, RZM, nzf, nsrc;
};

std::string yz_prelude(const sf_ctx *c, const YZShape &sh, const std::vector<DetectSource> &srcs)
{
    std::string p;
    p += "#define SFD_WY " + std::to_string(sh.WY) + "\n";
    p += "#define SFD_WZ " + std::to_string(sh.WZ) + "\n";
    p += "#define SFD_THREADS " + std::to_string(sh.threads) + "\n";
    p += "#define SFD_NSRC " + std::to_string(sh.nsrc) + "\n";
    p += "#define SFD_NZF " + std::to_string(sh.nzf) + "\n";
    p += "#define SFD_RYM " + std::to_string(sh.RYM) + "\n";
    p += "#define SFD_RZM " + std::to_string(sh.RZM) + "\n";
    p += "#define SFD_HZ " + std::to_string(sh.HZ) + "\n";
    p += "#define SFD_CH " + std::to_string(sh.CH) + "\n";
    p += "#define SFD_SROW " + std::to_string(sh.SROW) + "\n";
    p += "#define SFD_UROW " + std::to_string(sh.UROW) + "\n";
    /* output rows per y-filter task: 4 (default), or 8 (half the tasks, fewer
     * slab reads per output) */
    p += "#define SFD_PY " + std::to_string(env_int("SF_PY", 4) == 8 ? 8 : 4) + "\n";
    p += std::string("typedef ") + storage_ctype(c->cfg.storage) + " sfd_t;\n";
    p += "#define SFD_SOURCES(X)";
    for (size_t i = 0; i < srcs.size(); ++i) {
        int rz[4] = {0, 0, 0, 0};
        for (size_t f = 0; f < srcs[i].filters.size(); ++f) rz[f] = c->filt[srcs[i].filters[f]].rz;
        p += " X(" + std::to_string(i) + ", " + std::to_string(srcs[i].ry) + ", " +
             std::to_string(srcs[i].filters.size()) + ", " + std::to_string(rz[0]) + ", " +
             std::to_string(rz[1]) + ", " + std::to_string(rz[2]) + ", " + std::to_string(rz[3]) + ")";
    }
    p += "\n";
    return p;
}

/* y/z taps parameter block: gy[nsrc][RYM+1], gz[nsrc][nzf][RZM+1] by |offset| */
std::vector<float> yz_taps(const sf_ctx *c, const YZShape &sh, const std::vector<DetectSource> &srcs)
{
    std::vector<float> t(sh.nsrc * (sh.RYM + 1) + sh.nsrc * sh.nzf * (sh.RZM + 1), 0.f);
    for (size_t i = 0; i < srcs.size(); ++i) {
        const Filt &f0 = c->filt[srcs[i].filters[0]];
        for (int j = 0; j <= srcs[i].ry; ++j) t[i * (sh.RYM + 1) + j] = f0.gxy[f0.rxy + j];
        for (size_t q = 0; q < srcs[i].filters.size(); ++q) {
            const Filt &f = c->filt[srcs[i].filters[q]];
            float *g = &t[sh.nsrc * (sh.RYM + 1) + (i * sh.nzf + q) * (sh.RZM + 1)];
            for (int j = 0; j <= f.rz; ++j) g[j] = f.gz[f.rz + j];
        }
    }
    return t;
}

void yz_common_shape(const sf_ctx *c, YZShape &sh, int rym, int rzm)
{
    const size_t eb = c->ebytes;
    const int vec = (int)(16 / eb);               /* elements per 16-byte chunk */
    if (c->cfg.nz % vec == 0) sh.CH = vec;
    else if (eb == 4 && c->cfg.nz % 2 == 0) sh.CH = 2;
    else if (eb == 4) sh.CH = 1;
    else if (c->cfg.nz % 4 == 0) sh.CH = 4;       /* 8-byte chunks of 16-bit */
    else if (c->cfg.nz % 2 == 0) sh.CH = 2;       /* 4-byte chunks of 16-bit */
    else sh.CH = 0;                               /* element loads */
    const int hzq = std::max(4, sh.CH);
    sh.HZ = (rzm + hzq - 1) / hzq * hzq;
    sh.RYM = rym;
    sh.RZM = rzm;
    const int uw = sh.WZ + 2 * sh.HZ;
    sh.UROW = odd_quad_stride(uw + 4);
    if (eb == 4) sh.SROW = odd_quad_stride(uw + 4);
    else sh.SROW = (int)align_up((size_t)uw + 4, 8);
}

/* ------------------------------------------------------- sf_filter ----- */
sf_status build_filter(sf_ctx *c, int fi, Launch *L)
{
    const Filt &f = c->filt[fi];
    YZShape sh{};
    sh.WY = 32;
    sh.WZ = 64;
    sh.threads = sh.WY * sh.WZ / 8;
    sh.nzf = 1;
    sh.nsrc = 1;
    yz_common_shape(c, sh, f.rxy, f.rz);
    std::vector<DetectSource> srcs{DetectSource{f.slot, f.rxy, {fi}}};
    const size_t slab_bytes = align_up((size_t)(sh.WY + 2 * sh.RYM) * sh.SROW * c->ebytes, 128);
    const size_t u_bytes = f.rxy > 0 ? (size_t)sh.WY * sh.UROW * 4 : 0;
    std::string p = "#define SF_KERNEL_FILTER 1\n" + yz_prelude(c, sh, srcs);
    p += "#define SFD_P 8\n";
    p += std::string("#define SFD_X2 ") + (env_int("SF_NO_X2", 0) ? "0" : "1") + "\n";
    p += "#define SFD_OFF_U " + std::to_string(slab_bytes) + "\n";
    std::string err;
    sf_status s = jit_kernel(p, "sf_yz_filter", c->device, &L->kernel, err);
    if (s != SF_OK) return fail(c, s, "filter kernel: %s", err.c_str());
    L->smem = slab_bytes + u_bytes;
    if (L->smem > 48 * 1024 && (s = set_smem(c, L->kernel, L->smem)) != SF_OK) return s;
    L->block = dim3(sh.threads);
    L->grid = dim3((unsigned)c->cfg.nx, (unsigned)((c->cfg.ny + sh.WY - 1) / sh.WY),
                   (unsigned)((c->cfg.nz + sh.WZ - 1) / sh.WZ));
    c->ftaps[fi] = yz_taps(c, sh, srcs);
    return SF_OK;
}

/* ------------------------------------------------------- sf_detect ----- */
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
    });
    return fn;
}

/* Tiled 3D tensor map of a cube [x][y][z] with box {srow, WY + 2 RY, 1}. */
bool encode_map_dims(const sf_ctx *c, const void *base, long long nx, long long ny, long long nz,
                     int srow, int ry, CUtensorMap *out, long long zstride = -1)
{
    /* rows zstride elements apart (default nz); columns past nz read as zero */
    if (zstride < 0) zstride = nz;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const CUtensorMapDataType dt = c->cfg.storage == SF_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                   : c->cfg.storage == SF_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                               : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t dims[3] = {(cuuint64_t)nz, (cuuint64_t)ny, (cuuint64_t)nx};
    const cuuint64_t strides[2] = {(cuuint64_t)(zstride * (long long)c->ebytes),
                                   (cuuint64_t)(ny * zstride * (long long)c->ebytes)};
    const cuuint32_t box[3] = {(cuuint32_t)srow, (cuuint32_t)(c->cfg.wy + 2 * ry), 1u};
    const cuuint32_t es[3] = {1u, 1u, 1u};
    return enc(out, dt, 3, const_cast<void *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

/* the detect path's maps: rows zs apart in the padded layout */
bool encode_map(const sf_ctx *c, const void *base, int ry, CUtensorMap *out)
{
    return encode_map_dims(c, base, c->cfg.nx, c->cfg.ny, c->cfg.nz, c->dSROW, ry, out,
                           c->dpad ? c->zs : c->cfg.nz);
}

/* the detect path's copy of the cube (padded layout), else nullptr */
const void *padded_copy(const sf_ctx *c)
{
    return c->dpad ? (const char *)c->scratch + c->xy_sigma.size() * c->cube_bytes : nullptr;
}

/* Shape, shared-memory layout and parameter blocks of the window code (the
 * stand-alone window kernel and the persistent kernel share it). */
struct WindowPlan {
    std::vector<DetectSource> srcs;
    YZShape sh{};
    int P = 8, minb = 3, nzf = 1, rym = 0, rzm = 0, threads = 0;
    bool any_y = false;
    size_t off_s0 = 0, off_s1 = 0, off_u = 0, off_pm = 0, off_mk = 0, off_rd = 0, off_th = 0,
           off_fl = 0, off_mb = 0, smem = 0;
    std::string prelude;        /* SFD_* definitions without the kernel selector */
    std::vector<float> taps;    /* sfd_taps parameter block */
};

/* inputs of the window code: the cube (sigma_xy = 0) first, then the scratch slots */
std::vector<DetectSource> window_sources(const sf_ctx *c)
{
    std::vector<std::pair<int, std::vector<int>>> groups;   /* slot, filters */
    auto add = [&](int slot, int fi) {
        for (auto &gr : groups)
            if (gr.first == slot) { gr.second.push_back(fi); return; }
        groups.push_back({slot, {fi}});
    };
    for (int i = 0; i < (int)c->filt.size(); ++i)
        if (c->filt[i].slot < 0) add(-1, i);
    for (int i = 0; i < (int)c->filt.size(); ++i)
        if (c->filt[i].slot >= 0) add(c->filt[i].slot, i);
    std::vector<DetectSource> srcs;
    for (auto &gr : groups)
        for (size_t i = 0; i < gr.second.size(); i += SF_MAX_NZF) {
            DetectSource d;
            d.slot = gr.first;
            d.ry = gr.first < 0 ? 0 : c->xy_radius[gr.first];
            d.filters.assign(gr.second.begin() + i,
                             gr.second.begin() + std::min(gr.second.size(), i + (size_t)SF_MAX_NZF));
            srcs.push_back(d);
        }
    return srcs;
}

/* CH: elements per cp.async copy; tma_shape: halo and row pitch usable by TMA.
 * Returns false when the window shape cannot be tiled by the window code. */
bool make_window_plan(const sf_ctx *c, int P, int minb, int CH, bool tma_shape, WindowPlan &wp,
                      int weighted = -1)
{
    const sf_config &g = c->cfg;
    if (g.wy % 8 != 0 || g.wz % 32 != 0 || g.wx > 64 || g.wz % (4 * P) != 0) return false;
    const long long threads = (long long)g.wy * g.wz / P;
    if (threads < 32 || threads > 1024) return false;
    wp.srcs = window_sources(c);
    if (weighted >= 0) {
        /* Eq. 1: each input becomes a (denominator, numerator) pair */
        std::vector<DetectSource> pairs;
        for (const DetectSource &d : wp.srcs) {
            DetectSource den = d;
            den.den = true;
            pairs.push_back(den);
            pairs.push_back(d);
        }
        wp.srcs.swap(pairs);
    }
    if ((int)wp.srcs.size() > SF_MAX_SRC) return false;
    wp.P = P;
    wp.minb = minb;
    wp.threads = (int)threads;
    for (auto &d : wp.srcs) {
        wp.rym = std::max(wp.rym, d.ry);
        wp.any_y |= d.ry > 0;
        wp.nzf = std::max(wp.nzf, (int)d.filters.size());
        for (int fi : d.filters) wp.rzm = std::max(wp.rzm, c->filt[fi].rz);
    }
    YZShape &sh = wp.sh;
    sh.WY = g.wy;
    sh.WZ = g.wz;
    sh.threads = (int)threads;
    sh.nzf = wp.nzf;
    sh.nsrc = (int)wp.srcs.size();
    sh.CH = CH;
    const int vec = (int)(16 / c->ebytes);
    const int hzq = std::max(std::max(4, CH), tma_shape ? vec : 1);
    sh.HZ = (wp.rzm + hzq - 1) / hzq * hzq;
    sh.RYM = wp.rym;
    sh.RZM = wp.rzm;
    const int uw = sh.WZ + 2 * sh.HZ;
    sh.UROW = odd_quad_stride(uw + 4);
    sh.SROW = c->ebytes == 4 ? odd_quad_stride(uw + 4) : (int)align_up((size_t)uw + 4, 8);
    const int nwarp = (int)threads / 32;
    const int nw = g.wz / 32;
    size_t off = 0;
    const size_t slab = align_up((size_t)(sh.WY + 2 * wp.rym) * sh.SROW * c->ebytes, 128);
    wp.off_s0 = off;
    off += slab;
    wp.off_s1 = off;
    off += slab;
    wp.off_u = off;
    off += wp.any_y ? align_up((size_t)sh.WY * sh.UROW * 4, 128) : 0;
    wp.off_pm = off;
    off += align_up((size_t)g.wx * nwarp * wp.nzf * 4, 16);
    wp.off_mk = off;
    off += align_up((size_t)g.wx * g.wy * nw * 4, 16);
    wp.off_rd = off;
    off += align_up((size_t)nwarp * wp.nzf * 3 * (c->cfg.stats_fp64 ? 8 : 4), 16);
    wp.off_th = off;
    off += align_up((size_t)wp.nzf * 4, 16);
    wp.off_fl = off;
    off += 16;
    wp.off_mb = off;
    off += 16;
    wp.smem = off + 128;   /* the kernels align their base to 128 bytes */
    if (wp.smem > kSmemLimit) return false;
    std::string p = yz_prelude(c, sh, wp.srcs);
    p += "#define SFD_P " + std::to_string(P) + "\n";
    p += "#define SFD_WX " + std::to_string(g.wx) + "\n";
    /* resident CTAs per SM the register allocation must allow */
    p += "#define SFD_MINB " + std::to_string(minb) + "\n";
    /* z-pass thread layout: whole rows per warp where the tile allows it */
    if (env_int("SF_ZMAP", 1) == 1 && 32 % (g.wz / P) == 0) p += "#define SFD_ZMAP 1\n";
    /* packed FP32 pairs (fma/add/mul .f32x2) for the y and z filters */
    p += std::string("#define SFD_X2 ") + (env_int("SF_NO_X2", 0) ? "0" : "1") + "\n";
    p += "#define SFD_OFF_SLAB0 " + std::to_string(wp.off_s0) + "\n";
    p += "#define SFD_OFF_SLAB1 " + std::to_string(wp.off_s1) + "\n";
    p += "#define SFD_OFF_U " + std::to_string(wp.off_u) + "\n";
    p += "#define SFD_OFF_PMAX " + std::to_string(wp.off_pm) + "\n";
    p += "#define SFD_OFF_MASK " + std::to_string(wp.off_mk) + "\n";
    p += "#define SFD_OFF_RED " + std::to_string(wp.off_rd) + "\n";
    p += "#define SFD_OFF_THR " + std::to_string(wp.off_th) + "\n";
    p += "#define SFD_OFF_FLAGS " + std::to_string(wp.off_fl) + "\n";
    p += "#define SFD_OFF_MBAR " + std::to_string(wp.off_mb) + "\n";
    /* three-input max and warp-reduced plane maxima (SF_NO_FASTMAX=1: shuffles) */
    if (env_int("SF_NO_FASTMAX", 0)) p += "#define SFD_FASTMAX 0\n";
    if (weighted >= 0) p += "#define SFD_WEIGHTED 1\n";
    if (c->cfg.stats_fp64) p += "#define SFD_STATS64 1\n";
    if (c->cfg.std_ddof) p += "#define SFD_DDOF 1\n";
    wp.prelude = p;
    wp.taps = yz_taps(c, sh, wp.srcs);
    if (weighted == 1) {
        /* the printed denominator of Eq. 1 sums w alone: unit taps */
        for (size_t i = 0; i < wp.srcs.size(); ++i) {
            if (!wp.srcs[i].den) continue;
            for (int j = 0; j <= wp.srcs[i].ry; ++j) wp.taps[i * (sh.RYM + 1) + j] = 1.f;
            for (size_t q = 0; q < wp.srcs[i].filters.size(); ++q) {
                float *gz = &wp.taps[sh.nsrc * (sh.RYM + 1) + (i * sh.nzf + q) * (sh.RZM + 1)];
                for (int j = 0; j <= c->filt[wp.srcs[i].filters[q]].rz; ++j) gz[j] = 1.f;
            }
        }
    }
    return true;
}

/* elements per cp.async copy for rows of nz elements */
int copy_chunk(size_t ebytes, long long nz)
{
    const int vec = (int)(16 / ebytes);
    if (nz % vec == 0) return vec;
    if (ebytes == 4) return nz % 2 == 0 ? 2 : 1;
    if (nz % 4 == 0) return 4;
    if (nz % 2 == 0) return 2;
    return 0;
}

/* TMA needs 16-byte row pitches and boxes of at most 256 elements per axis */
bool tma_usable(const sf_ctx *c, const WindowPlan &wp, long long nz)
{
    const int vec = (int)(16 / c->ebytes);
    return nz % vec == 0 && wp.sh.SROW <= 256 && c->cfg.wy + 2 * wp.rym <= 256 &&
           tensor_map_encoder() != nullptr && env_int("SF_NO_TMA", 0) == 0;
}

/* A tiled 3D map of a 16-bit cube with the 128-byte swizzle and box {64,
 * rows, planes}: four planes of a window's rows straight into the K-major
 * layout the tensor-core MMAs read (rows = WY, planes = 4), or one plane's
 * slab of KY rows, read as an MN-major operand (rows = KY, planes = 1). */
bool encode_map_tc(const sf_ctx *c, const void *base, int rows, int planes, CUtensorMap *out)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const CUtensorMapDataType dt = c->cfg.storage == SF_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                             : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const long long zs = c->dpad ? c->zs : c->cfg.nz;   /* rows zs apart in the padded layout */
    const cuuint64_t dims[3] = {(cuuint64_t)c->cfg.nz, (cuuint64_t)c->cfg.ny, (cuuint64_t)c->cfg.nx};
    const cuuint64_t strides[2] = {(cuuint64_t)(zs * (long long)c->ebytes),
                                   (cuuint64_t)(c->cfg.ny * zs * (long long)c->ebytes)};
    const cuuint32_t box[3] = {64u, (cuuint32_t)rows, (cuuint32_t)planes};
    const cuuint32_t es[3] = {1u, 1u, 1u};
    return enc(out, dt, 3, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

/* byte offset of element (row, k) of a K-major tile with 128-byte rows and the
 * 128-byte swizzle (16-byte chunk index XOR row % 8, 8-row atoms of 1 KB) */
size_t sw128_offset(int row, int kbyte)
{
    return (size_t)(row / 8) * 1024 + (size_t)(row % 8) * 128 + (size_t)(((kbyte / 16) ^ (row % 8)) & 7) * 16 +
           (size_t)(kbyte % 16);
}

/* v as two 16-bit parts of the storage type, v ~ hi + lo */
void split16(const sf_ctx *c, float v, uint16_t *hi, uint16_t *lo)
{
    if (c->cfg.storage == SF_BF16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
        std::memcpy(hi, &h, 2);
        std::memcpy(lo, &l, 2);
    } else {
        const __half h = __float2half_rn(v);
        const __half l = __float2half_rn(v - __half2float(h));
        std::memcpy(hi, &h, 2);
        std::memcpy(lo, &l, 2);
    }
}

/* The window kernel with the y and z filters on the tensor cores, for 16-bit
 * storage: window 32 x 32 x 64, at most two spectral filters per input, the
 * z radius with its halo within the 64-column Toeplitz tile, y radius <= 16,
 * rows TMA-able.  Leaves c->use_tc false when the shape does not qualify. */
sf_status plan_detect_tc(sf_ctx *c)
{
    const sf_config &g = c->cfg;
    c->use_tc = false;
    /* TMA row strides: nz a multiple of 8, or the padded layout */
    const long long zs = c->dpad ? c->zs : g.nz;
    if (c->ebytes != 2 || g.wy != 32 || g.wz != 64 || g.wx > 64 || zs % 8 != 0 ||
        tensor_map_encoder() == nullptr)
        return SF_OK;
    WindowPlan wp;
    if (!make_window_plan(c, 8, 2, c->dpad ? 8 : copy_chunk(c->ebytes, g.nz), true, wp)) return SF_OK;
    if (wp.nzf > 2 || wp.sh.HZ + wp.rzm > 48 || wp.rym > 16 || !tma_usable(c, wp, zs)) return SF_OK;
    const int nsrc = (int)wp.srcs.size();
    const int HZ = wp.sh.HZ;
    auto ky_of = [&](int ry) { return (g.wy + 2 * ry + 15) / 16 * 16; };
    const int kym = ky_of(wp.rym);
    /* tap tiles: the z tiles of the distinct spectral filters, a y tile per
     * y-filtered input; zt / yt index them */
    std::vector<std::vector<float>> zkeys;
    std::vector<int> zt((size_t)nsrc * wp.nzf, 0), yt(nsrc, -1);
    int nyt = 0;
    for (int i = 0; i < nsrc; ++i) {
        for (size_t q = 0; q < wp.srcs[i].filters.size(); ++q) {
            const Filt &f = c->filt[wp.srcs[i].filters[q]];
            std::vector<float> key(f.gz.begin(), f.gz.end());
            int id = -1;
            for (size_t u = 0; u < zkeys.size(); ++u)
                if (zkeys[u] == key) id = (int)u;
            if (id < 0) {
                id = (int)zkeys.size();
                zkeys.push_back(key);
            }
            zt[(size_t)i * wp.nzf + q] = id;
        }
        if (wp.srcs[i].ry > 0) yt[i] = nyt++;
    }
    const int nzt = (int)zkeys.size();
    /* z tiles: the kernel's z MMAs take 32 outputs (pair p of 16-output
     * tiles) per MMA against rows t0 .. t0+31 of a tall Toeplitz tile
     * Tt[t][kk] = g[kk - t + C] (16 columns, no swizzle), t0 = 32p + HZ + C -
     * 16S for the K-slices S of the pair; C and the rows follow the kernel's
     * sft_zc / sft_zt0 */
    auto zlo = [&](int r, int pp) { return (32 * pp + HZ - r) / 16; };
    auto zhi = [&](int r, int pp) { return (32 * pp + 31 + HZ + r) / 16; };
    auto zc = [&](int r) {
        const int m = std::max(16 * zhi(r, 0) - HZ, 16 * zhi(r, 1) - 32 - HZ);
        return m <= 0 ? 0 : (m + 7) / 8 * 8;
    };
    int zrows = 0;
    for (int u = 0; u < nzt; ++u) {
        const int rz = ((int)zkeys[u].size() - 1) / 2;
        for (int pp = 0; pp < 2; ++pp)
            zrows = std::max(zrows, 32 * pp + HZ + zc(rz) - 16 * zlo(rz, pp) + 32);
    }
    zrows = (zrows + 15) / 16 * 16;   /* the y tile after the z tiles stays 1024-aligned */
    const size_t zpart = (size_t)zrows * 32;
    const size_t zbytes = (size_t)nzt * 2 * zpart, ybytes = (size_t)std::max(1, nyt) * 2 * 4096;
    const size_t tile_bytes = zbytes + ybytes;
    /* the parameter block: tiles, then zt[nsrc][nzf] and yt[nsrc] as int32 */
    c->tcb.assign(tile_bytes + sizeof(int32_t) * ((size_t)nsrc * wp.nzf + nsrc), 0);
    const float scale = 1024.f;   /* 2^10: the z taps' low parts stay normal */
    for (int u = 0; u < nzt; ++u) {
        const std::vector<float> &gz = zkeys[u];
        const int rz = ((int)gz.size() - 1) / 2, C = zc(rz);
        for (int t = 0; t < zrows; ++t)
            for (int kk = 0; kk < 16; ++kk) {
                const int o = kk - t + C;
                const float v = (o >= -rz && o <= rz) ? gz[rz + o] * scale : 0.f;
                uint16_t hi, lo;
                split16(c, v, &hi, &lo);
                /* 8-row groups of two 8 x 16-byte core matrices (k 0-7, 8-15) */
                const size_t off = (size_t)(t / 8) * 256 + (size_t)(kk / 8) * 128 + (size_t)(t % 8) * 16 + (size_t)(kk % 8) * 2;
                std::memcpy(&c->tcb[((size_t)u * 2 + 0) * zpart + off], &hi, 2);
                std::memcpy(&c->tcb[((size_t)u * 2 + 1) * zpart + off], &lo, 2);
            }
    }
    for (int i = 0; i < nsrc; ++i) {
        if (yt[i] < 0) continue;
        const Filt &f = c->filt[wp.srcs[i].filters[0]];
        const int ry = wp.srcs[i].ry;
        for (int n = 0; n < 32; ++n)
            for (int k = 0; k < 64; ++k) {
                const int o = k - n - ry;
                const float v = (o >= -ry && o <= ry) ? f.gxy[f.rxy + o] : 0.f;
                uint16_t hi, lo;
                split16(c, v, &hi, &lo);
                std::memcpy(&c->tcb[zbytes + ((size_t)yt[i] * 2 + 0) * 4096 + sw128_offset(n, 2 * k)], &hi, 2);
                std::memcpy(&c->tcb[zbytes + ((size_t)yt[i] * 2 + 1) * 4096 + sw128_offset(n, 2 * k)], &lo, 2);
            }
    }
    {
        int32_t *ix = reinterpret_cast<int32_t *>(&c->tcb[tile_bytes]);
        for (size_t j = 0; j < zt.size(); ++j) ix[j] = zt[j];
        for (int i = 0; i < nsrc; ++i) ix[zt.size() + i] = yt[i];
    }
    /* every CTA stages the tiles from device memory (coalesced, through L2):
     * read from the parameter block their per-thread addresses would
     * serialise in the constant cache */
    cudaFree(c->d_tct);
    c->d_tct = nullptr;
    if (cudaMalloc(&c->d_tct, tile_bytes) != cudaSuccess ||
        cudaMemcpy(c->d_tct, c->tcb.data(), tile_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(c, SF_ECUDA, "tap tile upload failed");
    /* shared memory (from a 1024-aligned base) */
    size_t off = 0;
    const size_t offA = off;
    off += 2 * 128 * 128;
    const size_t offT = off;
    /* the z tiles, and one y-tile slot the kernel fills per input */
    off += align_up(zbytes + (nyt > 0 ? (size_t)2 * 4096 : 0), 1024);
    const size_t offS = off;
    /* three slab buffers; inputs with sigma_xy = 0 use the region as a
     * second A tile (two 16 KB atoms) */
    bool any_ry0 = false;
    for (int i = 0; i < nsrc; ++i) any_ry0 |= wp.srcs[i].ry == 0;
    off += std::max<size_t>((size_t)3 * 2 * kym * 128, any_ry0 ? 2 * 16384 : 0);
    const size_t offP = off;
    off += align_up((size_t)g.wx * wp.nzf * 4, 16);
    const size_t offM = off;
    off += align_up((size_t)g.wx * g.wy * 2 * 4, 16);
    const size_t offR = off;
    off += align_up((size_t)8 * 3 * (g.stats_fp64 ? 8 : 4), 16);
    const size_t offTh = off;
    off += 16;
    const size_t offF = off;
    off += 16;
    const size_t offMB = off;
    off += 128;   /* 3 slab, 2 A-tile, 2 z and 2 y barriers */
    const size_t smem = off + 1024;
    if (smem > kSmemLimit) return SF_OK;
    std::string p = "#define SF_KERNEL_TC 1\n" + wp.prelude + "#define SFD_TMA 1\n";
    p += "#define SFT_OFF_A " + std::to_string(offA) + "\n";
    p += "#define SFT_OFF_T " + std::to_string(offT) + "\n";
    p += "#define SFT_OFF_SLAB " + std::to_string(offS) + "\n";
    p += "#define SFT_OFF_PMAX " + std::to_string(offP) + "\n";
    p += "#define SFT_OFF_MASK " + std::to_string(offM) + "\n";
    p += "#define SFT_OFF_RED " + std::to_string(offR) + "\n";
    p += "#define SFT_OFF_THR " + std::to_string(offTh) + "\n";
    p += "#define SFT_OFF_FLAGS " + std::to_string(offF) + "\n";
    p += "#define SFT_OFF_MBAR " + std::to_string(offMB) + "\n";
    p += "#define SFT_NZT " + std::to_string(nzt) + "\n";
    p += "#define SFT_ZROWS " + std::to_string(zrows) + "\n";
    p += "#define SFT_NYT " + std::to_string(nyt) + "\n";
    p += std::string("#define SFT_BF16 ") + (g.storage == SF_BF16 ? "1" : "0") + "\n";
    std::string err;
    sf_status s = jit_kernel(p, "sf_window_tc", c->device, &c->tclaunch.kernel, err);
    if (s != SF_OK) return fail(c, s, "tensor-core window kernel: %s", err.c_str());
    c->tclaunch.smem = smem;
    if ((s = set_smem(c, c->tclaunch.kernel, smem)) != SF_OK) return s;
    c->tclaunch.block = dim3(256);
    c->tclaunch.grid = dim3((unsigned)c->nwin);
    c->tcmaps.assign(nsrc, CUtensorMap{});
    for (int i = 0; i < nsrc; ++i) {
        if (wp.srcs[i].slot >= 0 &&
            !encode_map_tc(c, (const char *)c->scratch + (size_t)wp.srcs[i].slot * c->cube_bytes,
                           ky_of(wp.srcs[i].ry), 1, &c->tcmaps[i]))
            return fail(c, SF_ECUDA, "tensor map encoding failed");
        /* the padded copy of the cube: A boxes of four planes, fixed */
        if (wp.srcs[i].slot < 0 && c->dpad && !encode_map_tc(c, padded_copy(c), g.wy, 4, &c->tcmaps[i]))
            return fail(c, SF_ECUDA, "tensor map encoding failed");
    }
    c->use_tc = true;
    return SF_OK;
}

/* The fused window kernel: one CTA per statistics window (see sf_kernels.cuh). */
sf_status plan_detect(sf_ctx *c)
{
    const sf_config &g = c->cfg;
    c->fused = false;
    int P = 8;
    const int penv = env_int("SF_WP", 0);
    if ((penv == 8 || penv == 16) && g.wz % (4 * penv) == 0) P = penv;
    const int minb = std::max(1, std::min(8, env_int("SF_WMINB", 3)));
    WindowPlan wp;
    /* rows that are not 16-byte multiples: the padded layout when the window
     * code can take TMA slabs at all (SF_NO_PAD=1: element copies instead) */
    bool tma = false;
    for (int attempt = 0; attempt < 2; ++attempt) {
        c->dpad = attempt == 0 && c->zs != g.nz && !c->xlaunch_p.empty() && env_int("SF_NO_PAD", 0) == 0;
        wp = WindowPlan{};
        const int ch = c->dpad ? (int)(16 / c->ebytes) : copy_chunk(c->ebytes, g.nz);
        if (!make_window_plan(c, P, minb, ch, true, wp)) {
            if (c->dpad) continue;
            return SF_OK;
        }
        tma = tma_usable(c, wp, c->dpad ? c->zs : g.nz);
        if (tma || !c->dpad) break;
    }
    std::string p = "#define SF_KERNEL_DETECT 1\n" + wp.prelude;
    p += std::string("#define SFD_TMA ") + (tma ? "1" : "0") + "\n";
    std::string err;
    sf_status s = jit_kernel(p, "sf_window_detect", c->device, &c->dlaunch.kernel, err);
    if (s != SF_OK) return fail(c, s, "window kernel: %s", err.c_str());
    c->dlaunch.smem = wp.smem;
    if (wp.smem > 48 * 1024 && (s = set_smem(c, c->dlaunch.kernel, wp.smem)) != SF_OK) return s;
    c->dlaunch.block = dim3((unsigned)wp.threads);
    c->dlaunch.grid = dim3((unsigned)c->nwin);
    c->dsrc = wp.srcs;
    c->dSROW = wp.sh.SROW;
    c->dtma = tma;
    c->dnzf = wp.nzf;
    c->dP = P;
    c->dthreads = wp.threads;
    c->dHZ = wp.sh.HZ;
    c->dCH = wp.sh.CH;
    c->dUROW = wp.sh.UROW;
    c->dRYM = wp.rym;
    c->dRZM = wp.rzm;
    c->dtaps = wp.taps;
    c->dmaps.assign(wp.srcs.size(), CUtensorMap{});
    if (tma)
        for (size_t i = 0; i < wp.srcs.size(); ++i) {
            /* scratch inputs, and in the padded layout the cube's copy */
            const void *base = wp.srcs[i].slot >= 0
                                   ? (const void *)((const char *)c->scratch + (size_t)wp.srcs[i].slot * c->cube_bytes)
                                   : padded_copy(c);
            if (base && !encode_map(c, base, wp.srcs[i].ry, &c->dmaps[i]))
                return fail(c, SF_ECUDA, "tensor map encoding failed");
        }
    c->fused = true;
    if (env_int("SF_NO_TC", 0) == 0 && (s = plan_detect_tc(c)) != SF_OK) return s;
    return SF_OK;
}

/* ------------------------------------------------- persistent form --- */
void free_persist(sf_ctx *c)
{
    if (c->gpending && c->gdone) cudaEventSynchronize(c->gdone);
    c->gpending = false;
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    if (c->gdone) cudaEventDestroy(c->gdone);
    cudaFree(c->d_units);
    cudaFree(c->d_items);
    cudaFree(c->d_maps);
    cudaFree(c->d_ctr);
    cudaFree(c->d_xcubes);
    cudaFreeHost(c->h_units);
    cudaFreeHost(c->h_maps);
    cudaFreeHost(c->h_xcubes);
    c->d_xcubes = c->h_xcubes = nullptr;
    c->gexec = nullptr;
    c->gstream = nullptr;
    c->gdone = nullptr;
    c->d_units = c->h_units = nullptr;
    c->d_items = nullptr;
    c->d_maps = c->h_maps = nullptr;
    c->d_ctr = nullptr;
    c->units.clear();
    c->unit_cube.clear();
    c->pready = false;
}

/* Plan, compile and capture the persistent kernel for c->cubes. */
sf_status plan_persist(sf_ctx *c, const sf_ctx::PersistPlan &pp)
{
    free_persist(c);
    const sf_config &g = c->cfg;
    const int nxy = (int)c->xy_sigma.size();
    if (nxy > SF_MAX_XOUT) return fail(c, SF_EINVAL, "the persistent form takes at most %d distinct sigma_xy", SF_MAX_XOUT);
    /* copies for cubes that cannot use TMA: the largest chunk all their rows
     * allow.  With the batched x pass, cubes with padded scratch rows (zs > nz)
     * read the padded scratch and a padded copy of themselves by TMA instead. */
    const int vec = (int)(16 / c->ebytes);
    const bool xbatch = pp.xbatch && nxy > 0;
    WindowPlan wp;
    bool any_pad = false;
    for (int attempt = 0; attempt < 2; ++attempt) {
        int ch = vec;
        for (const sf_ctx::Cube &q : c->cubes)
            if (q.nz % vec != 0 && !(attempt == 1 && xbatch && q.zs != q.nz))
                ch = std::min(ch, copy_chunk(c->ebytes, q.nz));
        wp = WindowPlan{};
        if (!make_window_plan(c, pp.P, pp.minb, ch, true, wp))
            return fail(c, SF_EINVAL, "window %dx%dx%d cannot be tiled by the persistent kernel (wy %% 8, "
                        "wz %% 32, wx <= 64)", g.wx, g.wy, g.wz);
        any_pad = false;
        for (sf_ctx::Cube &q : c->cubes) {
            q.pad = attempt == 1 && xbatch && q.zs != q.nz;
            any_pad |= q.pad;
            q.tma = q.pad || tma_usable(c, wp, q.nz);
            q.xv = (q.ny * q.nz) % 2 == 0 && c->ebytes == 4 ? 2 : 1;
        }
        /* padding pays only where the window code can take TMA at all */
        if (attempt == 1 || !xbatch || !tma_usable(c, wp, vec)) break;
        bool want = false;
        for (const sf_ctx::Cube &q : c->cubes) want |= q.zs != q.nz;
        if (!want) break;
    }
    int r[4] = {0, 0, 0, 0}, rm = 0;
    for (int i = 0; i < nxy; ++i) {
        r[i] = c->xy_radius[i];
        rm = std::max(rm, r[i]);
    }
    /* padded cubes: one more x-pass output, the identity (radius 0, tap 1),
     * which writes the padded copy of the cube exactly */
    std::string xp = "#define SFX_NOUT " + std::to_string(std::max(1, nxy + (any_pad ? 1 : 0))) + "\n";
    for (int i = 0; i < 4; ++i) xp += "#define SFX_R" + std::to_string(i) + " " + std::to_string(r[i]) + "\n";
    xp += "#define SFX_RM " + std::to_string(rm) + "\n";
    xp += "#define SFX_PF " + std::to_string(pp.pf) + "\n";
    xp += std::string("typedef ") + storage_ctype(g.storage) + " sfx_t;\n";
    std::string p = "#define SF_KERNEL_PERSIST 1\n" + wp.prelude + "#define SFD_TMA 1\n" + xp;
    if (xbatch) p += "#define SFP_XITEMS 0\n";
    std::string err;
    sf_status st = jit_kernel(p, "sf_persist", c->device, &c->plaunch.kernel, err);
    if (st != SF_OK) return fail(c, st, "persistent kernel: %s", err.c_str());
    constexpr int kXbThreads = 128, kXbDepth = 8;
    if (xbatch) {
        /* the staged x pass of every cube in one launch, 16 bytes per slot */
        const std::string xb = "#define SF_KERNEL_XBATCH 1\n" + xp + "#define SFX_THREADS " +
                               std::to_string(kXbThreads) + "\n#define SFX_D " +
                               std::to_string(kXbDepth) + "\n";
        if ((st = jit_kernel(xb, "sf_xpass_batch", c->device, &c->xblaunch.kernel, err)) != SF_OK)
            return fail(c, st, "batched x pass: %s", err.c_str());
        c->xblaunch.block = dim3(kXbThreads);
        c->xblaunch.smem = (size_t)kXbDepth * kXbThreads * 2 * c->ebytes;
        if (c->xblaunch.smem > 48 * 1024 && (st = set_smem(c, c->xblaunch.kernel, c->xblaunch.smem)) != SF_OK)
            return st;
    }
    if (wp.smem > 48 * 1024 && (st = set_smem(c, c->plaunch.kernel, wp.smem)) != SF_OK) return st;
    int per_sm = 0, nsm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)c->plaunch.kernel,
                                                                  wp.threads, wp.smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "occupancy query");
    c->pp = pp;
    c->ptaps = wp.taps;
    std::vector<int> all;
    for (int i = 0; i < nxy; ++i) all.push_back(i);
    c->pxtaps = nxy ? xpass_taps(c, all) : std::vector<float>(1, 1.f);
    if (any_pad) {
        std::vector<float> id((size_t)rm + 1, 0.f);
        id[0] = 1.f;
        c->pxtaps.insert(c->pxtaps.end(), id.begin(), id.end());
    }
    c->psrc = wp.srcs;
    c->pnsrc = (int)wp.srcs.size();
    c->psrow = wp.sh.SROW;
    c->prym = wp.rym;

    /* units: each cube, or x-slabs of it (multiples of wx) */
    std::vector<int> unit_windows;
    for (size_t i = 0; i < c->cubes.size(); ++i) {
        const sf_ctx::Cube &q = c->cubes[i];
        long long slab = pp.slab > 0 ? ((long long)pp.slab + g.wx - 1) / g.wx * g.wx : q.nx;
        if (slab <= 0) slab = q.nx;
        for (long long x0 = 0; x0 < q.nx; x0 += slab) {
            sf_unit u{};
            u.x0 = x0;
            u.x1 = std::min(q.nx, x0 + slab);
            u.plane = q.ny * q.nz;
            u.xv = q.xv;
            u.lanes = u.plane / q.xv;
            u.tma = q.tma ? 1 : 0;
            u.map_base = (int)i * c->pnsrc;
            u.xlanes = pp.xlanes;
            u.n_xitems = nxy > 0 && !xbatch ? (int)((u.lanes + pp.xlanes - 1) / pp.xlanes) : 0;
            u.wx0 = (int)(x0 / g.wx);
            const int nwxu = (int)((u.x1 - x0 + g.wx - 1) / g.wx);
            c->units.push_back(u);
            c->unit_cube.push_back((int)i);
            unit_windows.push_back(nwxu * q.nwy * q.nwz);
        }
    }
    /* items: x items of unit k+1 come before the windows of unit k */
    std::vector<sf_item> items;
    const int nu = (int)c->units.size();
    auto push_x = [&](int u) {
        for (int j = 0; j < c->units[u].n_xitems; ++j) items.push_back(sf_item{u, 0, j, 0});
    };
    if (nu > 0) push_x(0);
    for (int u = 0; u < nu; ++u) {
        if (u + 1 < nu) push_x(u + 1);
        for (int j = 0; j < unit_windows[u]; ++j) items.push_back(sf_item{u, 1, j, 0});
    }
    c->n_items = (int)items.size();
    const size_t nmaps = c->cubes.size() * (size_t)c->pnsrc;
    if ((e = cudaMalloc(&c->d_units, sizeof(sf_unit) * nu)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_items, sizeof(sf_item) * std::max<size_t>(1, items.size()))) != cudaSuccess ||
        (e = cudaMalloc(&c->d_maps, sizeof(CUtensorMap) * std::max<size_t>(1, nmaps))) != cudaSuccess ||
        (e = cudaMalloc(&c->d_ctr, sizeof(int) * (1 + nu))) != cudaSuccess ||
        (e = cudaMallocHost(&c->h_units, sizeof(sf_unit) * nu)) != cudaSuccess ||
        (e = cudaMallocHost(&c->h_maps, sizeof(CUtensorMap) * std::max<size_t>(1, nmaps))) != cudaSuccess) {
        cudaGetLastError();
        free_persist(c);
        return fail(c, SF_ENOMEM, "persistent-form tables");
    }
    std::memset(c->h_maps, 0, sizeof(CUtensorMap) * std::max<size_t>(1, nmaps));
    long long xblocks = 0;
    if (xbatch) {
        const size_t nc = c->cubes.size();
        if ((e = cudaMalloc(&c->d_xcubes, sizeof(sf_xcube) * nc)) != cudaSuccess ||
            (e = cudaMallocHost(&c->h_xcubes, sizeof(sf_xcube) * nc)) != cudaSuccess) {
            cudaGetLastError();
            free_persist(c);
            return fail(c, SF_ENOMEM, "batched x-pass table");
        }
        /* per cube: lanes of two elements, or one where the y-z plane is odd */
        for (size_t i = 0; i < nc; ++i) {
            const sf_ctx::Cube &q = c->cubes[i];
            sf_xcube &xc = c->h_xcubes[i];
            std::memset(&xc, 0, sizeof(xc));
            const long long plane = q.ny * q.nz;
            /* padded rows: pairs only where a pair never straddles a row */
            xc.v = (q.pad ? q.nz % 2 == 0 : plane % 2 == 0) ? 2 : 1;
            xc.nz = q.nz;
            xc.ozs = q.pad ? q.zs : q.nz;
            xc.nx = q.nx;
            xc.x0 = 0;
            xc.x1 = q.nx;
            xc.plane = plane;
            xc.lanes = plane / xc.v;
            xc.block0 = (int)xblocks;
            xblocks += (xc.lanes + kXbThreads - 1) / kXbThreads;
        }
        if (xblocks > INT32_MAX) return fail(c, SF_EINVAL, "batched x pass: too many blocks");
        c->xblaunch.grid = dim3((unsigned)xblocks);
    }
    if (!items.empty() &&
        (e = cudaMemcpy(c->d_items, items.data(), sizeof(sf_item) * items.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(c, e, "item table");
    /* tensor maps of the scratch inputs (and of a padded cube's copy, the
     * slot after them) do not change between calls */
    for (size_t i = 0; i < c->cubes.size(); ++i) {
        const sf_ctx::Cube &q = c->cubes[i];
        if (!q.tma) continue;
        for (int sidx = 0; sidx < c->pnsrc; ++sidx) {
            const DetectSource &d = c->psrc[sidx];
            if (d.slot < 0 && !q.pad) continue;
            const int slot = d.slot < 0 ? nxy : d.slot;
            if (!encode_map_dims(c, (const char *)q.slots + (size_t)slot * q.slot_bytes, q.nx, q.ny, q.nz,
                                 c->psrow, d.ry, &c->h_maps[i * c->pnsrc + sidx], q.pad ? q.zs : q.nz))
                return fail(c, SF_ECUDA, "tensor map encoding failed");
        }
    }
    c->plaunch.block = dim3((unsigned)wp.threads);
    c->plaunch.grid = dim3((unsigned)std::max(1, std::min(per_sm * nsm, std::max(1, c->n_items))));
    c->plaunch.smem = wp.smem;

    /* capture: reset the counters, stage the tables, launch */
    if ((e = cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->gdone, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(c, e, "graph stream");
    sf_pargs pa{};
    pa.units = c->d_units;
    pa.items = c->d_items;
    pa.maps = c->d_maps;
    pa.head = c->d_ctr;
    pa.xdone = c->d_ctr + 1;
    pa.err = c->err_flag;
    pa.n_items = c->n_items;
    pa.xextra = xbatch ? 0 : c->stall_extra;
    pa.wait_ns = c->wait_ns;
    cudaGraph_t graph = nullptr;
    if ((e = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(c, e, "graph capture");
    cudaMemsetAsync(c->d_ctr, 0, sizeof(int) * (1 + nu), c->gstream);
    cudaMemcpyAsync(c->d_units, c->h_units, sizeof(sf_unit) * nu, cudaMemcpyHostToDevice, c->gstream);
    cudaMemcpyAsync(c->d_maps, c->h_maps, sizeof(CUtensorMap) * std::max<size_t>(1, nmaps),
                    cudaMemcpyHostToDevice, c->gstream);
    cudaError_t xe = cudaSuccess;
    if (xbatch) {
        cudaMemcpyAsync(c->d_xcubes, c->h_xcubes, sizeof(sf_xcube) * c->cubes.size(),
                        cudaMemcpyHostToDevice, c->gstream);
        sf_xbargs xa{};
        xa.cubes = c->d_xcubes;
        xa.n = (int)c->cubes.size();
        void *xargs[] = {&xa, c->pxtaps.data()};
        cudaLaunchConfig_t xl{};
        xl.gridDim = c->xblaunch.grid;
        xl.blockDim = c->xblaunch.block;
        xl.dynamicSmemBytes = c->xblaunch.smem;
        xl.stream = c->gstream;
        xe = cudaLaunchKernelExC(&xl, (const void *)c->xblaunch.kernel, xargs);
    }
    void *args[] = {&pa, c->ptaps.data(), c->pxtaps.data()};
    cudaLaunchConfig_t lc{};
    lc.gridDim = c->plaunch.grid;
    lc.blockDim = c->plaunch.block;
    lc.dynamicSmemBytes = c->plaunch.smem;
    lc.stream = c->gstream;
    cudaError_t le = cudaLaunchKernelExC(&lc, (const void *)c->plaunch.kernel, args);
    e = cudaStreamEndCapture(c->gstream, &graph);
    if (le != cudaSuccess) e = le;
    if (xe != cudaSuccess) e = xe;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(c, e, "persistent graph");
    c->pready = true;
    return SF_OK;
}

/* One replay of the persistent graph over the given cubes. */
sf_status run_persist(sf_ctx *c, const void *const *cubes, uint32_t *const *masks, float *const *means,
                      float *const *stds, cudaStream_t st)
{
    if (!c->pready) return fail(c, SF_ESTATE, "persistent form not planned");
    cudaError_t e;
    if (c->gpending && (e = cudaEventSynchronize(c->gdone)) != cudaSuccess)
        return cuda_fail(c, e, "previous batch");
    c->gpending = false;
    const sf_config &g = c->cfg;
    for (size_t u = 0; u < c->units.size(); ++u) {
        const int i = c->unit_cube[u];
        const sf_ctx::Cube &q = c->cubes[i];
        sf_unit h = c->units[u];
        sf_dargs &a = h.args;
        for (int sidx = 0; sidx < c->pnsrc; ++sidx) {
            const DetectSource &d = c->psrc[sidx];
            /* a padded cube's own input is its copy, the slot after the scratch cubes */
            const int slot = d.slot < 0 && q.pad ? (int)c->xy_sigma.size() : d.slot;
            a.src[sidx] = slot < 0 ? cubes[i] : (const void *)((const char *)q.slots + (size_t)slot * q.slot_bytes);
            for (size_t f = 0; f < d.filters.size(); ++f) a.fidx[sidx][f] = d.filters[f];
        }
        a.mask = masks[i];
        a.mean = means ? means[i] : nullptr;
        a.stdv = stds ? stds[i] : nullptr;
        if ((a.mean == nullptr) != (a.stdv == nullptr)) return fail(c, SF_EINVAL, "mean/std of cube %d", i);
        a.nx = q.nx;
        a.ny = q.ny;
        a.nz = q.nz;
        a.nw32 = q.nw32;
        a.nwx = q.nwx;
        a.nwy = q.nwy;
        a.nwz = q.nwz;
        a.nwin = q.nwin;
        a.k = g.k;
        a.err = c->err_flag;
        a.wait_ns = c->wait_ns;
        h.xsrc = cubes[i];
        for (int k = 0; k < SF_MAX_XOUT; ++k)
            h.xdst[k] = k < (int)c->xy_sigma.size() ? (void *)((char *)q.slots + (size_t)k * q.slot_bytes) : nullptr;
        c->h_units[u] = h;
    }
    if (c->h_xcubes) {
        for (size_t i = 0; i < c->cubes.size(); ++i) {
            const sf_ctx::Cube &q = c->cubes[i];
            sf_xcube &xc = c->h_xcubes[i];
            xc.src = cubes[i];
            const int nout = (int)c->xy_sigma.size() + (q.pad ? 1 : 0);   /* the copy: the identity output */
            for (int k = 0; k < SF_MAX_XOUT; ++k)
                xc.dst[k] = k < nout ? (void *)((char *)q.slots + (size_t)k * q.slot_bytes) : nullptr;
        }
    }
    for (size_t i = 0; i < c->cubes.size(); ++i) {
        const sf_ctx::Cube &q = c->cubes[i];
        if (!q.tma || q.pad) continue;
        for (int sidx = 0; sidx < c->pnsrc; ++sidx)
            if (c->psrc[sidx].slot < 0 &&
                !encode_map_dims(c, cubes[i], q.nx, q.ny, q.nz, c->psrow, c->psrc[sidx].ry,
                                 &c->h_maps[i * c->pnsrc + sidx]))
                return fail(c, SF_ECUDA, "tensor map encoding of cube %zu failed", i);
    }
    if ((e = cudaGraphLaunch(c->gexec, st)) != cudaSuccess) return cuda_fail(c, e, "graph launch");
    if ((e = cudaEventRecord(c->gdone, st)) != cudaSuccess) return cuda_fail(c, e, "graph event");
    c->gpending = true;
    return SF_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

sf_status check_live(sf_ctx *c, bool sectioned_ok = false)
{
    if (!c) return SF_EINVAL;
    if (c->dead) return fail(c, SF_ESTATE, "context unusable after an earlier CUDA error");
    if (c->sectioned && !sectioned_ok) return fail(c, SF_EINVAL, "sectioned context: use sf_detect_host");
    return SF_OK;
}

/* the window kernel over windows [w0, w1) of the plain context's cube; for
 * an x slab inside the cube (sf_detect_slab) the window grid starts at plane
 * xorg, ends at plane nx_end and has nwx windows along x */
sf_status launch_windows(sf_ctx *c, const void *d_cube, uint32_t *d_mask, float *d_mean, float *d_std,
                         cudaStream_t st, int w0, int w1, long long xorg = 0, long long nx_end = -1,
                         int nwx = -1)
{
    sf_dargs da{};
    for (size_t i = 0; i < c->dsrc.size(); ++i) {
        const DetectSource &d = c->dsrc[i];
        /* the cube itself: the caller's buffer, or in the padded layout its
         * copy written by the x pass (whose map is fixed) */
        da.src[i] = d.slot < 0 ? (c->dpad ? padded_copy(c) : d_cube)
                               : (const void *)((const char *)c->scratch + (size_t)d.slot * c->cube_bytes);
        for (size_t q = 0; q < d.filters.size(); ++q) da.fidx[i][q] = d.filters[q];
        if (c->dtma && d.slot < 0 && !c->dpad && !encode_map(c, d_cube, d.ry, &c->dmaps[i]))
            return fail(c, SF_ECUDA, "tensor map encoding of the cube failed");
    }
    da.mask = d_mask;
    da.mean = d_mean;
    da.stdv = d_std;
    da.nx = nx_end >= 0 ? nx_end : c->cfg.nx;
    da.ny = c->cfg.ny;
    da.nz = c->cfg.nz;
    da.nw32 = c->nw32;
    da.nwx = nwx >= 0 ? nwx : c->nwx;
    da.nwy = c->nwy;
    da.nwz = c->nwz;
    da.nwin = da.nwx * c->nwy * c->nwz;
    da.k = c->cfg.k;
    da.err = c->err_flag;
    da.wait_ns = c->wait_ns;
    da.xorg = xorg;
    da.wid0 = w0;
    if (c->use_tc) {
        /* the cube's own A boxes, swizzled, per call */
        for (size_t i = 0; i < c->dsrc.size() && !c->dpad; ++i)
            if (c->dsrc[i].slot < 0 && !encode_map_tc(c, d_cube, c->cfg.wy, 4, &c->tcmaps[i]))
                return fail(c, SF_ECUDA, "tensor map encoding of the cube failed");
        Launch L = c->tclaunch;
        L.grid = dim3((unsigned)(w1 - w0));
        void *args[] = {&da, c->dtaps.data(), c->tcmaps.data(), c->tcb.data(), &c->d_tct};
        return launch(c, L, args, st, "tensor-core window kernel launch");
    }
    Launch L = c->dlaunch;
    L.grid = dim3((unsigned)(w1 - w0));
    void *args[] = {&da, c->dtaps.data(), c->dmaps.data()};
    return launch(c, L, args, st, "window kernel launch");
}

cudaEvent_t take_event(sf_ctx *c)
{
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

/* begin/end of a timed stage on stream st (no-ops unless profiling) */
struct StageTimer {
    sf_ctx *c;
    int stage;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    StageTimer(sf_ctx *c_, int stage_, cudaStream_t st_) : c(c_), stage(stage_), st(st_)
    {
        if (c->prof && (a = take_event(c)) != nullptr) cudaEventRecord(a, st);
    }
    void done(int launches)
    {
        if (!a) return;
        cudaEvent_t b = take_event(c);
        if (!b) { c->pool.push_back(a); a = nullptr; return; }
        cudaEventRecord(b, st);
        c->recs.push_back(sf_ctx::Rec{stage, a, b, launches});
        a = nullptr;
    }
    ~StageTimer()
    {
        if (a) c->pool.push_back(a);
    }
};

}  // namespace

/* message for sf_last_error(NULL) from entry points that have no context */
void sf_set_global_error(const char *msg)
{
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_create_error = msg;
}

/* ============================================================ C ABI ===== */
extern "C" {

const char *sf_status_str(sf_status s)
{
    switch (s) {
    case SF_OK: return "SF_OK";
    case SF_EINVAL: return "SF_EINVAL";
    case SF_ENOMEM: return "SF_ENOMEM";
    case SF_EBUDGET: return "SF_EBUDGET";
    case SF_ECUDA: return "SF_ECUDA";
    case SF_ETIMEOUT: return "SF_ETIMEOUT";
    case SF_ESTATE: return "SF_ESTATE";
    case SF_EJIT: return "SF_EJIT";
    case SF_ECANCELED: return "SF_ECANCELED";
    }
    return "SF_UNKNOWN";
}

const char *sf_last_error(const sf_ctx *ctx)
{
    if (ctx) return ctx->err.c_str();
    std::lock_guard<std::mutex> lk(g_err_mu);
    static thread_local std::string copy;
    copy = g_create_error;
    return copy.c_str();
}

/* Plain context (n == 0: the cube of cfg) or batched context (n cubes of dims). */
static sf_status create_impl(const sf_config *cfg_in, int32_t n, const int64_t *dims, sf_ctx **out)
{
    if (!out) return fail(nullptr, SF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg_in) return fail(nullptr, SF_EINVAL, "cfg is NULL");
    sf_config g = *cfg_in;
    if (n < 0 || n > (1 << 20) || (n > 0 && !dims)) return fail(nullptr, SF_EINVAL, "batch of %d cubes", n);
    for (int i = 0; i < n; ++i)
        if (dims[3 * i] < 1 || dims[3 * i + 1] < 1 || dims[3 * i + 2] < 1 || dims[3 * i] > (1LL << 31) ||
            dims[3 * i + 1] > (1LL << 31) || dims[3 * i + 2] > (1LL << 31))
            return fail(nullptr, SF_EINVAL, "cube %d: dimensions must be in [1, 2^31]", i);
    if (n > 0) {
        g.nx = dims[0];
        g.ny = dims[1];
        g.nz = dims[2];
    }
    if (g.nx < 1 || g.ny < 1 || g.nz < 1)
        return fail(nullptr, SF_EINVAL, "cube dimensions must be >= 1 (got %lld x %lld x %lld)",
                    (long long)g.nx, (long long)g.ny, (long long)g.nz);
    if (g.nx > (1LL << 31) || g.ny > (1LL << 31) || g.nz > (1LL << 31))
        return fail(nullptr, SF_EINVAL, "cube dimension above 2^31");
    if (g.n_filters < 1 || g.n_filters > kMaxFilters || !g.filters)
        return fail(nullptr, SF_EINVAL, "n_filters must be in [1, %d] with a filter array", kMaxFilters);
    if (!(g.truncation > 0.f) || !std::isfinite(g.truncation))
        return fail(nullptr, SF_EINVAL, "truncation must be positive");
    if (g.wx < 1 || g.wy < 1 || g.wz < 1) return fail(nullptr, SF_EINVAL, "window sizes must be >= 1");
    if (!std::isfinite(g.k)) return fail(nullptr, SF_EINVAL, "k must be finite");
    if (g.storage != SF_F32 && g.storage != SF_F16 && g.storage != SF_BF16)
        return fail(nullptr, SF_EINVAL, "unknown storage dtype %d", g.storage);
    if (g.stats_fp64 != 0 && g.stats_fp64 != 1) return fail(nullptr, SF_EINVAL, "stats_fp64 must be 0 or 1");
    if (g.std_ddof != 0 && g.std_ddof != 1) return fail(nullptr, SF_EINVAL, "std_ddof must be 0 or 1");
    for (int i = 0; i < g.n_filters; ++i) {
        const sf_filter_spec &f = g.filters[i];
        if (!(f.sigma_xy >= 0.f) || !(f.sigma_z >= 0.f) || !std::isfinite(f.sigma_xy) ||
            !std::isfinite(f.sigma_z))
            return fail(nullptr, SF_EINVAL, "filter %d: sigmas must be finite and >= 0", i);
        if (radius_of(f.sigma_xy, g.truncation) > kMaxRadius || radius_of(f.sigma_z, g.truncation) > kMaxRadius)
            return fail(nullptr, SF_EINVAL, "filter %d: radius above %d", i, kMaxRadius);
    }
    int dev = g.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, SF_ECUDA, "no CUDA device");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || dev >= ndev)
        return fail(nullptr, SF_ECUDA, "CUDA device %d not available", dev);

    sf_ctx *c = new sf_ctx();
    c->cfg = g;
    c->cfg.filters = nullptr;
    c->device = dev;
    c->ebytes = storage_bytes(g.storage);
    c->nvox = g.nx * g.ny * g.nz;
    c->nw32 = (g.nz + 31) / 32;
    c->nwx = (int)((g.nx + g.wx - 1) / g.wx);
    c->nwy = (int)((g.ny + g.wy - 1) / g.wy);
    c->nwz = (int)((g.nz + g.wz - 1) / g.wz);
    c->nwin = c->nwx * c->nwy * c->nwz;
    for (int i = 0; i < g.n_filters; ++i) {
        Filt f;
        f.sxy = g.filters[i].sigma_xy;
        f.sz = g.filters[i].sigma_z;
        f.rxy = radius_of(f.sxy, g.truncation);
        f.rz = radius_of(f.sz, g.truncation);
        for (double v : gaussian_taps(f.sxy, f.rxy)) f.gxy.push_back((float)v);
        for (double v : gaussian_taps(f.sz, f.rz)) f.gz.push_back((float)v);
        if (f.rxy > 0) {
            int slot = -1;
            for (size_t s = 0; s < c->xy_sigma.size(); ++s)
                if (c->xy_sigma[s] == f.sxy) slot = (int)s;
            if (slot < 0) {
                slot = (int)c->xy_sigma.size();
                c->xy_sigma.push_back(f.sxy);
                c->xy_radius.push_back(f.rxy);
            }
            f.slot = slot;
        }
        c->filt.push_back(f);
    }

    DeviceGuard dg(dev);
    if (!dg.ok) {
        delete c;
        return fail(nullptr, SF_ECUDA, "cudaSetDevice(%d) failed", dev);
    }
    /* x pass shape: the widest vector that divides the y-z plane and keeps
     * the register ring (V * (2R+1+PF) floats) within about 96 registers */
    const long long plane = g.ny * g.nz;
    const int vmax = (int)(16 / c->ebytes);
    int rxm = 0;
    for (int r : c->xy_radius) rxm = std::max(rxm, r);
    c->xpf = env_int("SF_XPF", 2);
    /* staged form: input planes stream through xd shared-memory slots per
     * thread, so the register ring holds just the 2R+1 planes in use; 16
     * slots for 16-bit storage keep as many bytes in flight as 8 slots of
     * float32 (the tile workload's FP16 x pass: 0.35 ms against 0.44 ms) */
    c->xd = std::max(0, std::min(16, env_int("SF_XD", c->ebytes == 4 ? 8 : 16)));
    if (c->xd > 0 && c->xd < 3) c->xd = 3;
    const int ring = 2 * rxm + 1 + (c->xd > 0 ? 0 : c->xpf);
    c->xv = 1;
    for (int v = vmax; v >= 1; v /= 2)
        if (plane % v == 0 && (v == 1 || v * ring <= 96)) { c->xv = v; break; }
    const int xv_env = env_int("SF_XV", 0);
    if (xv_env > 0 && xv_env <= vmax && plane % xv_env == 0) c->xv = xv_env;
    /* cp.async copies 4, 8 or 16 bytes */
    if (c->xv * (int)c->ebytes < 4) c->xd = 0;
    const int xt_env = env_int("SF_XT", 128);
    c->xthreads = (xt_env == 64 || xt_env == 128 || xt_env == 256 || xt_env == 512) ? xt_env : 128;
    c->xseg = g.nx;
    const int nseg = env_int("SF_XSEG", 1);
    if (nseg > 1) c->xseg = (g.nx + nseg - 1) / nseg;
    {
        const long long vec = 16 / c->ebytes;
        c->zs = g.nz % vec != 0 ? (g.nz + vec - 1) / vec * vec : g.nz;
    }
    /* one scratch slot: sized for the padded z stride */
    c->cube_bytes = align_up((size_t)(g.nx * g.ny * c->zs) * c->ebytes, 256);
    sf_status s = SF_OK;
    {
        cudaError_t e = cudaMalloc(&c->err_flag, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(c->err_flag, 0, sizeof(int));
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return fail(nullptr, SF_ENOMEM, "error flag allocation failed");
        }
    }
    if (n > 0) {
        /* batched context: scratch of every cube in one allocation, one persistent plan */
        c->batch = true;
        size_t total = 0;
        for (int i = 0; i < n; ++i) {
            sf_ctx::Cube q{};
            q.nx = dims[3 * i];
            q.ny = dims[3 * i + 1];
            q.nz = dims[3 * i + 2];
            q.nw32 = (q.nz + 31) / 32;
            q.nwx = (int)((q.nx + g.wx - 1) / g.wx);
            q.nwy = (int)((q.ny + g.wy - 1) / g.wy);
            q.nwz = (int)((q.nz + g.wz - 1) / g.wz);
            q.nwin = q.nwx * q.nwy * q.nwz;
            /* rows that are not 16-byte multiples cannot be copied by TMA:
             * the batched x pass writes such a cube's scratch cubes, and a
             * copy of the cube itself, with rows padded to 16 bytes */
            const long long vec = 16 / c->ebytes;
            const size_t nxy = c->xy_sigma.size();
            q.zs = q.nz % vec != 0 && nxy > 0 && nxy < SF_MAX_XOUT ? (q.nz + vec - 1) / vec * vec : q.nz;
            q.slot_bytes = align_up((size_t)(q.nx * q.ny * q.zs) * c->ebytes, 256);
            total += q.slot_bytes * (nxy + (q.zs != q.nz ? 1 : 0));
            c->cubes.push_back(q);
        }
        if (total > 0) {
            cudaError_t e = cudaMalloc(&c->bscratch, total);
            if (e != cudaSuccess) {
                cudaGetLastError();
                s = fail(c, SF_ENOMEM, "batch scratch allocation of %zu bytes failed", total);
            }
        }
        size_t off = 0;
        for (sf_ctx::Cube &q : c->cubes) {
            q.slots = c->bscratch ? (char *)c->bscratch + off : nullptr;
            off += q.slot_bytes * (c->xy_sigma.size() + (q.zs != q.nz ? 1 : 0));
        }
        if (s == SF_OK) {
            sf_ctx::PersistPlan dp;
            dp.xbatch = true;   /* the default until sf_tune chooses */
            s = plan_persist(c, dp);
        }
        if (s != SF_OK) {
            {
                std::lock_guard<std::mutex> lk(g_err_mu);
                g_create_error = c->err;
            }
            sf_destroy(c);
            return s;
        }
        *out = c;
        return SF_OK;
    }
    const size_t nslot = c->xy_sigma.size() + (c->zs != g.nz ? 1 : 0);
    if (nslot > 0) {
        cudaError_t e = cudaMalloc(&c->scratch, c->cube_bytes * nslot);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return fail(nullptr, SF_ENOMEM, "scratch allocation of %zu bytes failed", c->cube_bytes * nslot);
        }
        for (size_t i = 0; i < c->xy_sigma.size(); i += SF_MAX_XOUT) {
            std::vector<int> slots;
            for (size_t j = i; j < std::min(c->xy_sigma.size(), i + SF_MAX_XOUT); ++j) slots.push_back((int)j);
            Launch L;
            if ((s = build_xpass(c, slots, &L)) != SF_OK) break;
            c->xgroups.push_back(slots);
            c->xlaunch.push_back(L);
        }
        /* the detect path's padded x passes: every slot and the copy; lanes
         * of two elements where nz is even (a lane stays within a row) */
        for (size_t i = 0; s == SF_OK && c->zs != g.nz && i < nslot; i += SF_MAX_XOUT) {
            std::vector<int> slots;
            for (size_t j = i; j < std::min(nslot, i + SF_MAX_XOUT); ++j) slots.push_back((int)j);
            Launch L;
            if ((s = build_xpass(c, slots, &L, g.nz % 2 == 0 ? std::min(2, c->xv) : 1)) != SF_OK) break;
            c->xgroups_p.push_back(slots);
            c->xlaunch_p.push_back(L);
        }
    }
    if (s == SF_OK) s = plan_detect(c);
    if (s != SF_OK) {
        {
            std::lock_guard<std::mutex> lk(g_err_mu);
            g_create_error = c->err;
        }
        sf_destroy(c);
        return s;
    }
    *out = c;
    return SF_OK;
}

sf_status sf_create(const sf_config *cfg, sf_ctx **out)
{
    return create_impl(cfg, 0, nullptr, out);
}

sf_status sf_create_batch(const sf_config *cfg, int32_t n, const int64_t *dims, sf_ctx **out)
{
    if (n < 1) {
        if (out) *out = nullptr;
        return fail(nullptr, SF_EINVAL, "a batch needs at least one cube");
    }
    return create_impl(cfg, n, dims, out);
}

sf_status sf_create_sectioned(const sf_config *cfg, int64_t section, sf_ctx **out)
{
    if (!out) return fail(nullptr, SF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, SF_EINVAL, "cfg is NULL");
    const sf_config &g = *cfg;
    if (g.wx < 1) return fail(nullptr, SF_EINVAL, "window sizes must be >= 1");
    if (section < 1 || section % g.wx != 0)
        return fail(nullptr, SF_EINVAL, "section must be a positive multiple of wx (%d)", g.wx);
    if (g.nx < 1 || g.nx > (1LL << 31)) return fail(nullptr, SF_EINVAL, "nx must be in [1, 2^31]");
    if (g.n_filters < 1 || g.n_filters > kMaxFilters || !g.filters)
        return fail(nullptr, SF_EINVAL, "n_filters must be in [1, %d] with a filter array", kMaxFilters);
    if (!(g.truncation > 0.f) || !std::isfinite(g.truncation))
        return fail(nullptr, SF_EINVAL, "truncation must be positive");
    int rxm = 0;
    for (int i = 0; i < g.n_filters; ++i) {
        const float sxy = g.filters[i].sigma_xy;
        if (!(sxy >= 0.f) || !std::isfinite(sxy)) return fail(nullptr, SF_EINVAL, "filter %d: sigmas must be finite and >= 0", i);
        rxm = std::max(rxm, radius_of(sxy, g.truncation));
    }
    /* halo: the largest x radius, rounded up to whole windows so that the
     * section context's windows fall on the cube's */
    const long long h = rxm > 0 ? ((long long)rxm + g.wx - 1) / g.wx * g.wx : 0;
    const bool one = g.nx <= section;
    const long long nsub[2] = {one ? g.nx : section + 2 * h,
                               one || g.nx % g.wx == 0 ? 0 : g.nx - (g.nx - 1) / section * section + h};
    sf_ctx *sub[2] = {nullptr, nullptr};
    for (int i = 0; i < 2; ++i) {
        if (!nsub[i]) continue;
        sf_config q = g;
        q.nx = nsub[i];
        sf_status s = create_impl(&q, 0, nullptr, &sub[i]);
        if (s != SF_OK) {
            if (sub[0]) sf_destroy(sub[0]);
            return s;
        }
    }
    sf_ctx *c = new sf_ctx();
    c->cfg = g;
    c->cfg.filters = nullptr;
    c->sectioned = true;
    c->device = sub[0]->device;
    c->ebytes = sub[0]->ebytes;
    c->nvox = g.nx * g.ny * g.nz;
    c->nw32 = sub[0]->nw32;
    c->sect_S = one ? g.nx : section;
    c->sect_h = one ? 0 : h;
    for (int i = 0; i < 2; ++i) {
        c->sub[i] = sub[i];
        c->sub_nx[i] = nsub[i];
    }
    DeviceGuard dg(c->device);
    const long long nmax = std::max(nsub[0], nsub[1]);
    const size_t in_bytes = (size_t)nmax * (size_t)(g.ny * g.nz) * c->ebytes;
    const size_t mask_bytes = (size_t)nmax * (size_t)(g.ny * c->nw32) * 4;
    for (int i = 0; i < 2; ++i) {
        if (cudaMalloc(&c->sbuf[i], in_bytes) != cudaSuccess ||
            cudaMalloc((void **)&c->smask[i], mask_bytes) != cudaSuccess) {
            cudaGetLastError();
            sf_destroy(c);
            return fail(nullptr, SF_ENOMEM, "section buffers (2 x %zu bytes)", in_bytes + mask_bytes);
        }
    }
    *out = c;
    return SF_OK;
}

sf_status sf_destroy(sf_ctx *c)
{
    if (!c) return SF_OK;
    DeviceGuard dg(c->device);
    cudaDeviceSynchronize();
    cudaGetLastError();
    free_persist(c);
    cudaFree(c->bscratch);
    cudaFree(c->scratch);
    cudaFree(c->filt_scratch);
    cudaFree(c->stat_scratch);
    cudaFree(c->host_cube);
    cudaFree(c->host_mask);
    cudaFree(c->err_flag);
    cudaFree(c->d_tct);
    for (cudaStream_t x : c->hcomp)
        if (x) cudaStreamDestroy(x);
    cudaFree(c->lscratch);
    cudaFree(c->wscratch);
    cudaFree(c->wstats);
    for (int i = 0; i < 2; ++i) {
        if (c->sub[i]) sf_destroy(c->sub[i]);
        cudaFree(c->sbuf[i]);
        cudaFree(c->smask[i]);
    }
    if (c->boxtwin) sf_destroy(c->boxtwin);
    if (c->gausstwin) sf_destroy(c->gausstwin);
    for (cudaStream_t x : c->hcopy)
        if (x) cudaStreamDestroy(x);
    if (c->hback) cudaStreamDestroy(c->hback);
    for (cudaEvent_t ev : c->hev) cudaEventDestroy(ev);
    for (const sf_ctx::Rec &r : c->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
    delete c;
    return SF_OK;
}

sf_status sf_taps(const sf_ctx *ctx, int32_t filter, int32_t axis, float *out, int32_t cap,
                  int32_t *radius)
{
    sf_ctx *c = const_cast<sf_ctx *>(ctx);
    if (!c) return SF_EINVAL;
    if (filter < 0 || filter >= (int)c->filt.size()) return fail(c, SF_EINVAL, "filter index %d", filter);
    if (axis < 0 || axis > 2) return fail(c, SF_EINVAL, "axis must be 0, 1 or 2");
    const Filt &f = c->filt[filter];
    const std::vector<float> &g = axis == 2 ? f.gz : f.gxy;
    if (radius) *radius = (int32_t)((g.size() - 1) / 2);
    if (out) {
        if (cap < (int32_t)g.size()) return fail(c, SF_EINVAL, "capacity %d below %zu taps", cap, g.size());
        std::memcpy(out, g.data(), g.size() * sizeof(float));
    }
    return SF_OK;
}

sf_status sf_window_grid(const sf_ctx *c, int32_t *nwx, int32_t *nwy, int32_t *nwz)
{
    if (!c) return SF_EINVAL;
    if (nwx) *nwx = c->nwx;
    if (nwy) *nwy = c->nwy;
    if (nwz) *nwz = c->nwz;
    return SF_OK;
}

sf_status sf_mask_words(const sf_ctx *c, int64_t *words)
{
    if (!c || !words) return SF_EINVAL;
    *words = c->cfg.nx * c->cfg.ny * c->nw32;
    return SF_OK;
}

sf_status sf_filter(sf_ctx *c, const void *d_cube, int32_t filter, float *d_filtered, void *stream)
{
    sf_status s = check_live(c);
    if (s != SF_OK) return s;
    if (c->batch) return fail(c, SF_EINVAL, "batched context: use sf_detect_batch");
    if (filter < 0 || filter >= (int)c->filt.size()) return fail(c, SF_EINVAL, "filter index %d", filter);
    if (!d_cube || !d_filtered) return fail(c, SF_EINVAL, "NULL buffer");
    if (!aligned16(d_cube) || !aligned16(d_filtered)) return fail(c, SF_EINVAL, "buffers must be 16-byte aligned");
    DeviceGuard dg(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const Filt &f = c->filt[filter];
    const void *src = d_cube;
    if (f.slot >= 0) {
        auto it = c->xsingle.find(f.slot);
        if (it == c->xsingle.end()) {
            Launch L;
            if ((s = build_xpass(c, {f.slot}, &L)) != SF_OK) return s;
            it = c->xsingle.emplace(f.slot, L).first;
        }
        if ((s = run_xpass(c, it->second, {f.slot}, d_cube, st)) != SF_OK) return s;
        src = (const char *)c->scratch + (size_t)f.slot * c->cube_bytes;
    }
    auto it = c->flaunch.find(filter);
    if (it == c->flaunch.end()) {
        Launch L;
        if ((s = build_filter(c, filter, &L)) != SF_OK) return s;
        it = c->flaunch.emplace(filter, L).first;
    }
    sf_fargs fa{};
    fa.src = src;
    fa.out = d_filtered;
    fa.nx = c->cfg.nx;
    fa.ny = c->cfg.ny;
    fa.nz = c->cfg.nz;
    std::vector<float> &taps = c->ftaps[filter];
    void *args[] = {&fa, taps.data()};
    return launch(c, it->second, args, st, "filter launch");
}

sf_status sf_stats(sf_ctx *c, const float *d_filtered, float *d_mean, float *d_std, void *stream)
{
    sf_status s = check_live(c);
    if (s != SF_OK) return s;
    if (c->batch) return fail(c, SF_EINVAL, "batched context: use sf_detect_batch");
    if (!d_filtered || !d_mean || !d_std) return fail(c, SF_EINVAL, "NULL buffer");
    DeviceGuard dg(c->device);
    const sf_config &g = c->cfg;
    cudaError_t e = sf_launch_stats(d_filtered, g.nx, g.ny, g.nz, g.wx, g.wy, g.wz, c->nwx, c->nwy,
                                    c->nwz, d_mean, d_std, c->cfg.stats_fp64, c->cfg.std_ddof,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stats launch");
    return SF_OK;
}

sf_status sf_threshold(sf_ctx *c, const float *d_filtered, const float *d_mean, const float *d_std,
                       uint32_t *d_mask, int32_t accumulate, void *stream)
{
    sf_status s = check_live(c);
    if (s != SF_OK) return s;
    if (c->batch) return fail(c, SF_EINVAL, "batched context: use sf_detect_batch");
    if (!d_filtered || !d_mean || !d_std || !d_mask) return fail(c, SF_EINVAL, "NULL buffer");
    DeviceGuard dg(c->device);
    const sf_config &g = c->cfg;
    cudaError_t e = sf_launch_threshold(d_filtered, g.nx, g.ny, g.nz, g.wx, g.wy, g.wz, c->nwy, c->nwz,
                                        d_mean, d_std, g.k, d_mask, accumulate ? 1 : 0,
                                        (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "threshold launch");
    return SF_OK;
}

sf_status sf_detect(sf_ctx *c, const void *d_cube, uint32_t *d_mask, float *d_mean, float *d_std,
                    void *stream)
{
    sf_status s = check_live(c);
    if (s != SF_OK) return s;
    if (!d_cube || !d_mask) return fail(c, SF_EINVAL, "NULL buffer");
    if ((d_mean == nullptr) != (d_std == nullptr))
        return fail(c, SF_EINVAL, "d_mean and d_std must both be NULL or both be set");
    if (!aligned16(d_cube)) return fail(c, SF_EINVAL, "cube must be 16-byte aligned");
    if (c->batch) return fail(c, SF_EINVAL, "batched context: use sf_detect_batch");
    DeviceGuard dg(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (c->use_persist) {
        StageTimer tp(c, 1, st);
        const void *cubes[1] = {d_cube};
        uint32_t *masks[1] = {d_mask};
        float *means[1] = {d_mean};
        float *stds[1] = {d_std};
        s = run_persist(c, cubes, masks, d_mean ? means : nullptr, d_std ? stds : nullptr, st);
        if (s == SF_OK) tp.done(1);
        return s;
    }
    {
        StageTimer tx(c, 0, st);
        const std::vector<Launch> &XL = c->dpad ? c->xlaunch_p : c->xlaunch;
        const std::vector<std::vector<int>> &XG = c->dpad ? c->xgroups_p : c->xgroups;
        for (size_t i = 0; i < XL.size(); ++i)
            if ((s = run_xpass(c, XL[i], XG[i], d_cube, st, 0, -1, c->dpad)) != SF_OK) return s;
        tx.done((int)XL.size());
    }
    StageTimer tf(c, 1, st);
    if (c->fused) {
        s = launch_windows(c, d_cube, d_mask, d_mean, d_std, st, 0, c->nwin);
        if (s == SF_OK) tf.done(1);
        return s;
    }
    /* composed path: per filter filter -> stats -> threshold (accumulate) */
    const size_t nwin = (size_t)c->nwin;
    if (!c->filt_scratch) {
        cudaError_t e = cudaMalloc(&c->filt_scratch, (size_t)c->nvox * 4);
        if (e == cudaSuccess) e = cudaMalloc(&c->stat_scratch, 2 * nwin * 4);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, SF_ENOMEM, "composed-path scratch allocation failed");
        }
    }
    for (int fi = 0; fi < (int)c->filt.size(); ++fi) {
        if ((s = sf_filter(c, d_cube, fi, c->filt_scratch, stream)) != SF_OK) return s;
        float *m = d_mean ? d_mean + fi * nwin : c->stat_scratch;
        float *sd = d_std ? d_std + fi * nwin : c->stat_scratch + nwin;
        if ((s = sf_stats(c, c->filt_scratch, m, sd, stream)) != SF_OK) return s;
        if ((s = sf_threshold(c, c->filt_scratch, m, sd, d_mask, fi > 0, stream)) != SF_OK) return s;
    }
    int nl = 0;
    for (const Filt &f : c->filt) nl += 3 + (f.slot >= 0 ? 1 : 0);
    tf.done(nl);
    return SF_OK;
}

sf_status sf_detect_slab(sf_ctx *c, const void *d_ext, int64_t halo, uint32_t *d_mask, float *d_mean,
                         float *d_std, void *stream)
{
    sf_status s = check_live(c);
    if (s != SF_OK) return s;
    if (!d_ext || !d_mask) return fail(c, SF_EINVAL, "NULL buffer");
    if ((d_mean == nullptr) != (d_std == nullptr))
        return fail(c, SF_EINVAL, "d_mean and d_std must both be NULL or both be set");
    if (!aligned16(d_ext)) return fail(c, SF_EINVAL, "cube must be 16-byte aligned");
    if (c->batch) return fail(c, SF_EINVAL, "batched context: slabs take a plain context");
    if (!c->fused) return fail(c, SF_EINVAL, "slabs need the fused window kernel (wy %% 8 == 0, wz %% 32 == 0)");
    int rxm = 0;
    for (int r : c->xy_radius) rxm = std::max(rxm, r);
    const long long S = c->cfg.nx - 2 * (long long)halo;
    if (halo < rxm || S < 1)
        return fail(c, SF_EINVAL, "halo %lld: needs >= %d planes and nx - 2 halo >= 1 (nx = %lld)",
                    (long long)halo, rxm, (long long)c->cfg.nx);
    DeviceGuard dg(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    {
        /* x pass of the slab's planes only; they read the halo planes */
        StageTimer tx(c, 0, st);
        const std::vector<Launch> &XL = c->dpad ? c->xlaunch_p : c->xlaunch;
        const std::vector<std::vector<int>> &XG = c->dpad ? c->xgroups_p : c->xgroups;
        for (size_t i = 0; i < XL.size(); ++i)
            if ((s = run_xpass(c, XL[i], XG[i], d_ext, st, halo, halo + S, c->dpad)) != SF_OK)
                return s;
        tx.done((int)XL.size());
    }
    StageTimer tf(c, 1, st);
    const int nwx = (int)((S + c->cfg.wx - 1) / c->cfg.wx);
    s = launch_windows(c, d_ext, d_mask, d_mean, d_std, st, 0, nwx * c->nwy * c->nwz, halo, halo + S, nwx);
    if (s == SF_OK) tf.done(1);
    return s;
}

sf_status sf_detect_batch(sf_ctx *c, const void *const *d_cubes, uint32_t *const *d_masks,
                          float *const *d_means, float *const *d_stds, void *stream)
{
    sf_status s = check_live(c);
    if (s != SF_OK) return s;
    if (!c->batch) return fail(c, SF_EINVAL, "not a batched context (sf_create_batch)");
    if (!d_cubes || !d_masks) return fail(c, SF_EINVAL, "NULL pointer array");
    if ((d_means == nullptr) != (d_stds == nullptr))
        return fail(c, SF_EINVAL, "d_means and d_stds must both be NULL or both be set");
    for (size_t i = 0; i < c->cubes.size(); ++i) {
        if (!d_cubes[i] || !d_masks[i]) return fail(c, SF_EINVAL, "cube %zu: NULL buffer", i);
        if (!aligned16(d_cubes[i])) return fail(c, SF_EINVAL, "cube %zu must be 16-byte aligned", i);
    }
    DeviceGuard dg(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    StageTimer tp(c, 1, st);
    s = run_persist(c, d_cubes, d_masks, d_means, d_stds, st);
    if (s == SF_OK) tp.done(1);
    return s;
}

extern "C++" {
namespace {
/* milliseconds per call of fn on stream st (1 warm-up, reps timed) */
template <class F>
float time_calls(sf_ctx *c, cudaStream_t st, int reps, F fn, sf_status *s)
{
    *s = fn();
    if (*s != SF_OK) return -1.f;
    cudaEvent_t a = take_event(c), b = take_event(c);
    if (!a || !b) {
        *s = fail(c, SF_ECUDA, "events");
        return -1.f;
    }
    cudaEventRecord(a, st);
    for (int i = 0; i < reps && *s == SF_OK; ++i) *s = fn();
    cudaEventRecord(b, st);
    float ms = -1.f;
    if (*s == SF_OK && cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
        ms /= reps;
    c->pool.push_back(a);
    c->pool.push_back(b);
    return ms;
}
}  // namespace
}

sf_status sf_tune(sf_ctx *c, const void *const *d_cubes, uint32_t *const *d_masks, void *stream)
{
    sf_status s = check_live(c);
    if (s != SF_OK) return s;
    if (!d_cubes || !d_masks) return fail(c, SF_EINVAL, "NULL pointer array");
    DeviceGuard dg(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const bool prof = c->prof;
    c->prof = false;
    std::string rep = "[";
    float best = 1e30f;
    int best_kind = -1;   /* -1: two-kernel path, else index into cands */
    std::vector<sf_ctx::PersistPlan> cands;
    const long long maxnx = c->batch ? 0 : c->cfg.nx;
    {
        /* x pass as one batched launch, then the windows */
        sf_ctx::PersistPlan q;
        q.xbatch = true;
        cands.push_back(q);
    }
    for (int slab : {0, 128, 256}) {
        if (!c->batch && slab > 0 && slab >= maxnx) continue;
        for (int xl : {1024, 4096}) {
            sf_ctx::PersistPlan q;
            q.slab = slab;
            q.xlanes = xl;
            cands.push_back(q);
        }
    }
    if (!c->batch) {
        /* the two-kernel path is the first candidate of a plain context */
        c->use_persist = false;
        const float ms = time_calls(c, st, 3, [&] { return sf_detect(c, d_cubes[0], d_masks[0], nullptr, nullptr, stream); }, &s);
        if (s != SF_OK) { c->prof = prof; return s; }
        rep += "{\"path\": \"x pass + window kernel\", \"ms\": " + std::to_string(ms) + "}";
        best = ms;
        c->cubes.clear();
        sf_ctx::Cube q{};
        q.nx = c->cfg.nx;
        q.ny = c->cfg.ny;
        q.nz = c->cfg.nz;
        q.nw32 = c->nw32;
        q.nwx = c->nwx;
        q.nwy = c->nwy;
        q.nwz = c->nwz;
        q.nwin = c->nwin;
        q.zs = q.nz;
        q.slot_bytes = c->cube_bytes;
        q.slots = c->scratch;
        c->cubes.push_back(q);
    }
    for (size_t k = 0; k < cands.size(); ++k) {
        if ((s = plan_persist(c, cands[k])) != SF_OK) break;
        const float ms = time_calls(c, st, 3, [&] {
            return run_persist(c, d_cubes, d_masks, nullptr, nullptr, st);
        }, &s);
        if (s != SF_OK) break;
        if (rep.size() > 1) rep += ", ";
        if (cands[k].xbatch)
            rep += "{\"path\": \"batched x pass + persistent windows\", \"ms\": " + std::to_string(ms) + "}";
        else
            rep += "{\"path\": \"persistent\", \"slab\": " + std::to_string(cands[k].slab) +
                   ", \"x_lanes_per_item\": " + std::to_string(cands[k].xlanes) + ", \"ms\": " +
                   std::to_string(ms) + "}";
        if (ms > 0.f && ms < best) {
            best = ms;
            best_kind = (int)k;
        }
    }
    rep += "]";
    c->tune_report = rep;
    if (s == SF_OK) {
        if (best_kind >= 0) {
            s = plan_persist(c, cands[best_kind]);
            c->use_persist = !c->batch;
        } else {
            free_persist(c);
            c->use_persist = false;
        }
    }
    if (s == SF_OK && (s = sf_synchronize(c, stream)) != SF_OK) {
        c->prof = prof;
        return s;
    }
    c->prof = prof;
    return s;
}

sf_status sf_tune_report(const sf_ctx *c, char *buf, int32_t cap)
{
    if (!c || !buf || cap < 1) return SF_EINVAL;
    std::snprintf(buf, (size_t)cap, "%s", c->tune_report.c_str());
    return (int)c->tune_report.size() < cap ? SF_OK : SF_EINVAL;
}

sf_status sf_profile_enable(sf_ctx *c, int32_t enable)
{
    if (!c) return SF_EINVAL;
    c->prof = enable != 0;
    return SF_OK;
}

sf_status sf_profile_read(sf_ctx *c, double *ms, int64_t *launches, int32_t n_stages)
{
    if (!c || n_stages < 0 || (n_stages > 0 && (!ms || !launches))) return SF_EINVAL;
    DeviceGuard dg(c->device);
    for (int i = 0; i < n_stages; ++i) {
        ms[i] = 0.0;
        launches[i] = 0;
    }
    sf_status s = SF_OK;
    for (const sf_ctx::Rec &r : c->recs) {
        cudaError_t e = cudaEventSynchronize(r.b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess && s == SF_OK) s = cuda_fail(c, e, "profile events");
        if (r.stage < n_stages) {
            ms[r.stage] += t;
            launches[r.stage] += r.launches;
        }
        c->pool.push_back(r.a);
        c->pool.push_back(r.b);
    }
    c->recs.clear();
    return s;
}

/* Sectioned detect from host buffers (Sec. 3.1: the cube is cut along x
 * into sections with a halo; Sec. 6: input overlapped with processing).
 * Section k covers planes [x0, x1) = [kS, min(nx, kS + S)); its context sees
 * planes [x0 - h, x0 - h + nsub), h a multiple of wx at least the largest x
 * radius, with zeros where that range leaves the cube, so the x pass of
 * planes [x0, x1) reads exactly the planes the whole-cube pass reads and the
 * statistics windows of [x0, x1) are the whole cube's.  Copies in, the
 * section's detect and the copy back of its mask rows run on three streams;
 * two section buffers alternate. */
sf_status detect_sections(sf_ctx *c, const void *h_cube, uint32_t *h_mask, void *stream)
{
    DeviceGuard dg(c->device);
    const sf_config &g = c->cfg;
    const size_t plane = (size_t)(g.ny * g.nz) * c->ebytes;
    const size_t mplane = (size_t)(g.ny * c->nw32) * 4;
    const long long nx = g.nx, S = c->sect_S, h = c->sect_h;
    const int K = (int)((nx + S - 1) / S);
    cudaError_t e;
    if (!c->hback) {
        if ((e = cudaStreamCreateWithFlags(&c->hcopy[0], cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&c->hcomp[0], cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&c->hback, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(c, e, "section streams");
    }
    while ((int)c->hev.size() < 3 * K + 2) {
        cudaEvent_t ev;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(c, e, "section events");
        c->hev.push_back(ev);
    }
    cudaStream_t st = (cudaStream_t)stream, cs = c->hcopy[0], ks = c->hcomp[0], bs = c->hback;
    cudaEvent_t *ev_in = &c->hev[0], *ev_run = &c->hev[K], *ev_out = &c->hev[2 * K];
    /* nothing may overtake earlier work on the caller's stream */
    cudaEventRecord(c->hev[3 * K], st);
    cudaStreamWaitEvent(cs, c->hev[3 * K], 0);
    cudaStreamWaitEvent(ks, c->hev[3 * K], 0);
    cudaStreamWaitEvent(bs, c->hev[3 * K], 0);
    sf_status s;
    long long plo = 0, phi = 0, porigin = 0;   /* planes held by the previous section's buffer */
    for (int k = 0; k < K; ++k) {
        const long long x0 = k * S, x1 = std::min(nx, x0 + S);
        const int b = k & 1;
        const int u = (K > 1 && x1 == nx && nx % g.wx != 0) ? 1 : 0;
        const long long origin = K == 1 ? 0 : x0 - h, nsub = c->sub_nx[u];
        const long long lo = std::max(0LL, origin), hi = std::min(nx, origin + nsub);
        char *buf = (char *)c->sbuf[b];
        /* the buffers of section k - 2 are free once its mask rows are back */
        if (k >= 2) cudaStreamWaitEvent(cs, ev_out[k - 2], 0);
        if (lo > origin && (e = cudaMemsetAsync(buf, 0, (size_t)(lo - origin) * plane, cs)) != cudaSuccess)
            return cuda_fail(c, e, "section padding");
        if (origin + nsub > hi &&
            (e = cudaMemsetAsync(buf + (size_t)(hi - origin) * plane, 0, (size_t)(origin + nsub - hi) * plane, cs)) !=
                cudaSuccess)
            return cuda_fail(c, e, "section padding");
        /* planes the previous section also holds (its right part, this one's
         * left halo) move device to device; only the rest crosses the host
         * link, so each plane does so once */
        const long long olo = k > 0 ? std::max(lo, plo) : lo, ohi = k > 0 ? std::min(hi, phi) : lo;
        auto h2d = [&](long long a, long long z) -> cudaError_t {
            if (z <= a) return cudaSuccess;
            return cudaMemcpyAsync(buf + (size_t)(a - origin) * plane, (const char *)h_cube + (size_t)a * plane,
                                   (size_t)(z - a) * plane, cudaMemcpyHostToDevice, cs);
        };
        if (ohi > olo) {
            const char *prev = (const char *)c->sbuf[b ^ 1];
            if ((e = cudaMemcpyAsync(buf + (size_t)(olo - origin) * plane, prev + (size_t)(olo - porigin) * plane,
                                     (size_t)(ohi - olo) * plane, cudaMemcpyDeviceToDevice, cs)) != cudaSuccess)
                return cuda_fail(c, e, "section overlap copy");
            if ((e = h2d(lo, olo)) != cudaSuccess || (e = h2d(ohi, hi)) != cudaSuccess)
                return cuda_fail(c, e, "section host-to-device copy");
        } else if ((e = h2d(lo, hi)) != cudaSuccess) {
            return cuda_fail(c, e, "section host-to-device copy");
        }
        plo = lo;
        phi = hi;
        porigin = origin;
        cudaEventRecord(ev_in[k], cs);
        cudaStreamWaitEvent(ks, ev_in[k], 0);
        if ((s = sf_detect(c->sub[u], buf, c->smask[b], nullptr, nullptr, ks)) != SF_OK)
            return fail(c, s, "section %d: %s", k, c->sub[u]->err.c_str());
        cudaEventRecord(ev_run[k], ks);
        cudaStreamWaitEvent(bs, ev_run[k], 0);
        if ((e = cudaMemcpyAsync((char *)h_mask + (size_t)x0 * mplane,
                                 (const char *)c->smask[b] + (size_t)(x0 - origin) * mplane,
                                 (size_t)(x1 - x0) * mplane, cudaMemcpyDeviceToHost, bs)) != cudaSuccess)
            return cuda_fail(c, e, "section device-to-host copy");
        cudaEventRecord(ev_out[k], bs);
    }
    cudaStreamWaitEvent(st, ev_out[K - 1], 0);
    return sf_synchronize(c, stream);
}

sf_status sf_detect_host(sf_ctx *c, const void *h_cube, uint32_t *h_mask, void *stream)
{
    sf_status s = check_live(c, true);
    if (s != SF_OK) return s;
    if (c->batch) return fail(c, SF_EINVAL, "batched context: use sf_detect_batch");
    if (!h_cube || !h_mask) return fail(c, SF_EINVAL, "NULL buffer");
    if (c->sectioned) return detect_sections(c, h_cube, h_mask, stream);
    DeviceGuard dg(c->device);
    const size_t plane = (size_t)(c->cfg.ny * c->cfg.nz) * c->ebytes;
    const size_t mplane = (size_t)(c->cfg.ny * c->nw32) * 4;
    const size_t cube = plane * (size_t)c->cfg.nx;
    const size_t mask = mplane * (size_t)c->cfg.nx;
    cudaError_t e;
    if (!c->host_cube) {
        e = cudaMalloc(&c->host_cube, cube);
        if (e == cudaSuccess) e = cudaMalloc((void **)&c->host_mask, mask);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, SF_ENOMEM, "device buffers for the host entry point");
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (c->use_persist || !c->fused) {
        /* whole-cube copies around one sf_detect */
        if ((e = cudaMemcpyAsync(c->host_cube, h_cube, cube, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(c, e, "host-to-device copy");
        if ((s = sf_detect(c, c->host_cube, c->host_mask, nullptr, nullptr, stream)) != SF_OK) return s;
        if ((e = cudaMemcpyAsync(h_mask, c->host_mask, mask, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_fail(c, e, "device-to-host copy");
        return sf_synchronize(c, stream);
    }
    /* Pipelined along x (Sec. 6: overlap input with processing): chunks of
     * whole window slabs go host-to-device on two copy streams; chunk k's x
     * pass starts once the chunks holding its planes and x halo have landed,
     * its window kernel follows on the same compute stream, and its mask rows
     * go back on a third stream.  Consecutive chunks alternate between two
     * compute streams, so one chunk's kernels fill the tail of the other's. */
    const long long wx = c->cfg.wx;
    const long long nx = c->cfg.nx;
    const long long nch = std::max(1, std::min(256, env_int("SF_HCHUNKS", 16)));
    long long S = (nx + nch - 1) / nch;
    S = std::max(wx, (S + wx - 1) / wx * wx);
    const int K = (int)((nx + S - 1) / S);
    int rxm = 0;
    for (int r : c->xy_radius) rxm = std::max(rxm, r);
    if (!c->hback) {
        for (int i = 0; i < 2; ++i)
            if ((e = cudaStreamCreateWithFlags(&c->hcopy[i], cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaStreamCreateWithFlags(&c->hcomp[i], cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_fail(c, e, "pipeline stream");
        if ((e = cudaStreamCreateWithFlags(&c->hback, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(c, e, "pipeline stream");
    }
    while ((int)c->hev.size() < 2 * K + 3) {
        cudaEvent_t ev;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(c, e, "pipeline events");
        c->hev.push_back(ev);
    }
    /* nothing may overtake earlier work on the caller's stream */
    cudaEventRecord(c->hev[2 * K], st);
    for (int i = 0; i < 2; ++i) {
        cudaStreamWaitEvent(c->hcopy[i], c->hev[2 * K], 0);
        cudaStreamWaitEvent(c->hcomp[i], c->hev[2 * K], 0);
    }
    cudaStreamWaitEvent(c->hback, c->hev[2 * K], 0);
    /* host-to-device chunks on one copy stream (SF_HCOPY=2: alternating two) */
    const int ncopy = env_int("SF_HCOPY", 1) == 2 ? 2 : 1;
    for (int k = 0; k < K; ++k) {
        const long long x0 = k * S, x1 = std::min(nx, x0 + S);
        cudaStream_t cs = c->hcopy[ncopy == 2 ? (k & 1) : 0];
        if ((e = cudaMemcpyAsync((char *)c->host_cube + (size_t)x0 * plane, (const char *)h_cube + (size_t)x0 * plane,
                                 (size_t)(x1 - x0) * plane, cudaMemcpyHostToDevice, cs)) != cudaSuccess)
            return cuda_fail(c, e, "host-to-device copy");
        cudaEventRecord(c->hev[k], cs);
    }
    int waited[2] = {-1, -1};
    for (int k = 0; k < K; ++k) {
        const long long x0 = k * S, x1 = std::min(nx, x0 + S);
        cudaStream_t ks = c->hcomp[k & 1];
        const int need = (int)(std::min(nx, x1 + rxm) - 1) / (int)S;
        for (int j = waited[k & 1] + 1; j <= need; ++j) cudaStreamWaitEvent(ks, c->hev[j], 0);
        waited[k & 1] = std::max(waited[k & 1], need);
        const std::vector<Launch> &XL = c->dpad ? c->xlaunch_p : c->xlaunch;
        const std::vector<std::vector<int>> &XG = c->dpad ? c->xgroups_p : c->xgroups;
        for (size_t i = 0; i < XL.size(); ++i)
            if ((s = run_xpass(c, XL[i], XG[i], c->host_cube, ks, x0, x1, c->dpad)) != SF_OK) return s;
        const int w0 = (int)(x0 / wx) * c->nwy * c->nwz;
        const int w1 = (int)((x1 + wx - 1) / wx) * c->nwy * c->nwz;
        if ((s = launch_windows(c, c->host_cube, c->host_mask, nullptr, nullptr, ks, w0, w1)) != SF_OK) return s;
        cudaEventRecord(c->hev[K + k], ks);
        cudaStreamWaitEvent(c->hback, c->hev[K + k], 0);
        if ((e = cudaMemcpyAsync((char *)h_mask + (size_t)x0 * mplane, (const char *)c->host_mask + (size_t)x0 * mplane,
                                 (size_t)(x1 - x0) * mplane, cudaMemcpyDeviceToHost, c->hback)) != cudaSuccess)
            return cuda_fail(c, e, "device-to-host copy");
    }
    /* the caller's stream resumes after the last copy back */
    cudaEventRecord(c->hev[2 * K + 1], c->hback);
    cudaStreamWaitEvent(st, c->hev[2 * K + 1], 0);
    return sf_synchronize(c, stream);
}

namespace {
sf_status local_check(sf_ctx *c, int sx, int sy, int sz)
{
    sf_status s = check_live(c);
    if (s != SF_OK) return s;
    if (c->batch) return fail(c, SF_EINVAL, "batched context: local statistics take one cube");
    if (sx < 0 || sy < 0 || sz < 0) return fail(c, SF_EINVAL, "box half-widths must be >= 0");
    if (sy > 64 || sz > 128) return fail(c, SF_EINVAL, "box half-widths sy <= 64 and sz <= 128");
    if (c->cfg.nx > 65535) return fail(c, SF_EINVAL, "local statistics take nx <= 65535");
    return SF_OK;
}

/* filtered cube (if `filtered`), P and Q scratch of the local statistics */
sf_status local_scratch(sf_ctx *c)
{
    if (c->lscratch) return SF_OK;
    const size_t cube = align_up((size_t)c->nvox * sizeof(float), 256);
    const cudaError_t e = cudaMalloc((void **)&c->lscratch, 3 * cube);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->lscratch = nullptr;
        return fail(c, SF_ENOMEM, "local-statistics scratch (%zu bytes)", 3 * cube);
    }
    return SF_OK;
}
}  // namespace

sf_status sf_local_stats(sf_ctx *c, const float *d_filtered, int32_t sx, int32_t sy, int32_t sz, float *d_mean,
                         float *d_std, void *stream)
{
    sf_status s = local_check(c, sx, sy, sz);
    if (s != SF_OK) return s;
    if (!d_filtered || !d_mean || !d_std) return fail(c, SF_EINVAL, "NULL buffer");
    DeviceGuard dg(c->device);
    if ((s = local_scratch(c)) != SF_OK) return s;
    const sf_config &g = c->cfg;
    const size_t cube = align_up((size_t)c->nvox * sizeof(float), 256) / sizeof(float);
    float *P = c->lscratch + cube, *Q = c->lscratch + 2 * cube;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (sf_local_is_narrow(sx, sy, sz)) {
        e = sf_launch_local_direct(d_filtered, g.nx, g.ny, g.nz, c->nw32, sx, sy, sz, g.k, d_mean, d_std,
                                   nullptr, 0, g.std_ddof, st);
    } else {
        e = sf_launch_local_yz(d_filtered, P, Q, g.nx, g.ny, g.nz, sy, sz, st);
        if (e == cudaSuccess)
            e = sf_launch_local_x(d_filtered, P, Q, g.nx, g.ny, g.nz, c->nw32, sx, sy, sz, g.k, d_mean, d_std,
                                  nullptr, 0, g.std_ddof, st);
    }
    return e == cudaSuccess ? SF_OK : cuda_fail(c, e, "local statistics launch");
}

sf_status sf_local_zscore(sf_ctx *c, const float *d_filtered, int32_t sx, int32_t sy, int32_t sz, float *d_z,
                          void *stream)
{
    sf_status s = local_check(c, sx, sy, sz);
    if (s != SF_OK) return s;
    if (!d_filtered || !d_z) return fail(c, SF_EINVAL, "NULL buffer");
    DeviceGuard dg(c->device);
    if ((s = local_scratch(c)) != SF_OK) return s;
    const sf_config &g = c->cfg;
    const size_t cube = align_up((size_t)c->nvox * sizeof(float), 256) / sizeof(float);
    float *P = c->lscratch + cube, *Q = c->lscratch + 2 * cube;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (sf_local_is_narrow(sx, sy, sz)) {
        e = sf_launch_local_direct(d_filtered, g.nx, g.ny, g.nz, c->nw32, sx, sy, sz, g.k, d_z, nullptr,
                                   nullptr, 3, g.std_ddof, st);
    } else {
        e = sf_launch_local_yz(d_filtered, P, Q, g.nx, g.ny, g.nz, sy, sz, st);
        if (e == cudaSuccess)
            e = sf_launch_local_x(d_filtered, P, Q, g.nx, g.ny, g.nz, c->nw32, sx, sy, sz, g.k, d_z, nullptr,
                                  nullptr, 3, g.std_ddof, st);
    }
    return e == cudaSuccess ? SF_OK : cuda_fail(c, e, "local z-score launch");
}

sf_status sf_local_detect(sf_ctx *c, const void *d_cube, int32_t sx, int32_t sy, int32_t sz, uint32_t *d_mask,
                          void *stream)
{
    sf_status s = local_check(c, sx, sy, sz);
    if (s != SF_OK) return s;
    if (!d_cube || !d_mask) return fail(c, SF_EINVAL, "NULL buffer");
    DeviceGuard dg(c->device);
    if ((s = local_scratch(c)) != SF_OK) return s;
    const sf_config &g = c->cfg;
    const size_t cube = align_up((size_t)c->nvox * sizeof(float), 256) / sizeof(float);
    float *F = c->lscratch, *P = c->lscratch + cube, *Q = c->lscratch + 2 * cube;
    cudaStream_t st = (cudaStream_t)stream;
    for (int f = 0; f < (int)c->filt.size(); ++f) {
        if ((s = sf_filter(c, d_cube, f, F, stream)) != SF_OK) return s;
        cudaError_t e;
        if (sf_local_is_narrow(sx, sy, sz)) {
            e = sf_launch_local_direct(F, g.nx, g.ny, g.nz, c->nw32, sx, sy, sz, g.k, nullptr, nullptr, d_mask,
                                       f == 0 ? 1 : 2, g.std_ddof, st);
        } else {
            e = sf_launch_local_yz(F, P, Q, g.nx, g.ny, g.nz, sy, sz, st);
            if (e == cudaSuccess)
                e = sf_launch_local_x(F, P, Q, g.nx, g.ny, g.nz, c->nw32, sx, sy, sz, g.k, nullptr, nullptr,
                                      d_mask, f == 0 ? 1 : 2, g.std_ddof, st);
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "local detect launch");
    }
    return SF_OK;
}

namespace {
sf_status weighted_check(sf_ctx *c, const float *d_cube, const float *d_w, int den)
{
    sf_status s = check_live(c);
    if (s != SF_OK) return s;
    if (c->batch) return fail(c, SF_EINVAL, "batched context: the weighted form takes one cube");
    if (c->cfg.storage != SF_F32) return fail(c, SF_EINVAL, "the weighted form takes float32 storage");
    if (den != 0 && den != 1) return fail(c, SF_EINVAL, "den must be 0 (sum f w) or 1 (sum w)");
    if (!d_cube || !d_w) return fail(c, SF_EINVAL, "NULL buffer");
    if (!aligned16(d_cube) || !aligned16(d_w)) return fail(c, SF_EINVAL, "buffers must be 16-byte aligned");
    return SF_OK;
}

sf_status weighted_scratch(sf_ctx *c, int den)
{
    if (!c->wscratch) {
        const size_t cube = align_up((size_t)c->nvox * sizeof(float), 256);
        cudaError_t e = cudaMalloc((void **)&c->wscratch, 3 * cube);
        if (e == cudaSuccess) e = cudaMalloc((void **)&c->wstats, 2 * sizeof(float) * (size_t)c->nwin);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaFree(c->wscratch);
            c->wscratch = nullptr;
            return fail(c, SF_ENOMEM, "weighted-form scratch (%zu bytes)", 3 * cube);
        }
    }
    if (den == 1 && !c->boxtwin) {
        /* same shape, bank radii and window; every tap 1 (a box sum) */
        sf_config cfg = c->cfg;
        std::vector<sf_filter_spec> specs;
        for (const Filt &f : c->filt) specs.push_back(sf_filter_spec{f.sxy, f.sz});
        cfg.filters = specs.data();
        cfg.device = c->device;
        sf_ctx *t = nullptr;
        sf_status s = create_impl(&cfg, 0, nullptr, &t);
        if (s != SF_OK) return fail(c, s, "box-tap twin context");
        for (Filt &f : t->filt) {
            std::fill(f.gxy.begin(), f.gxy.end(), 1.f);
            std::fill(f.gz.begin(), f.gz.end(), 1.f);
        }
        c->boxtwin = t;
    }
    return SF_OK;
}

/* a twin of the context (same shape, bank and window): its scratch cubes
 * hold the x-filtered weights of the fused Eq. 1 path */
sf_status weighted_gauss_twin(sf_ctx *c)
{
    if (c->gausstwin) return SF_OK;
    sf_config cfg = c->cfg;
    std::vector<sf_filter_spec> specs;
    for (const Filt &f : c->filt) specs.push_back(sf_filter_spec{f.sxy, f.sz});
    cfg.filters = specs.data();
    cfg.device = c->device;
    sf_ctx *t = nullptr;
    sf_status s = create_impl(&cfg, 0, nullptr, &t);
    if (s != SF_OK) return fail(c, s, "twin context");
    c->gausstwin = t;
    return SF_OK;
}

/* the fused Eq. 1 window kernel for denominator reading den, built once;
 * not ready when the window cannot be tiled (the composed path runs then) */
sf_status weighted_plan(sf_ctx *c, int den)
{
    sf_ctx::WPlan &W = c->wplan[den];
    if (W.tried) return SF_OK;
    W.tried = true;
    if (env_int("SF_WCOMPOSED", 0)) return SF_OK;
    const sf_config &g = c->cfg;
    WindowPlan wp;
    if (!make_window_plan(c, 8, 2, copy_chunk(c->ebytes, g.nz), true, wp, den)) return SF_OK;
    W.tma = tma_usable(c, wp, g.nz);
    std::string p = "#define SF_KERNEL_DETECT 1\n" + wp.prelude;
    p += std::string("#define SFD_TMA ") + (W.tma ? "1" : "0") + "\n";
    std::string err;
    sf_status s = jit_kernel(p, "sf_window_detect", c->device, &W.L.kernel, err);
    if (s != SF_OK) return fail(c, s, "weighted window kernel: %s", err.c_str());
    W.L.smem = wp.smem;
    if (wp.smem > 48 * 1024 && (s = set_smem(c, W.L.kernel, wp.smem)) != SF_OK) return s;
    W.L.block = dim3((unsigned)wp.threads);
    W.L.grid = dim3((unsigned)c->nwin);
    W.taps = wp.taps;
    W.srcs = wp.srcs;
    W.maps.assign(wp.srcs.size(), CUtensorMap{});
    W.ready = true;
    return SF_OK;
}

/* c = Eq. 1 for filter f of the bank, into out; p = d * w already formed */
sf_status weighted_one(sf_ctx *c, const float *p, const float *d_w, int f, int den, float *out, cudaStream_t st)
{
    const size_t cube = align_up((size_t)c->nvox * sizeof(float), 256) / sizeof(float);
    float *num = c->wscratch + cube, *dn = c->wscratch + 2 * cube;
    sf_status s = sf_filter(c, p, f, num, st);
    if (s != SF_OK) return s;
    sf_ctx *dc = den == 1 ? c->boxtwin : c;
    if ((s = sf_filter(dc, d_w, f, dn, st)) != SF_OK) return dc == c ? s : fail(c, s, "%s", dc->err.c_str());
    const cudaError_t e = sf_launch_w_ratio(num, dn, out, c->nvox, st);
    return e == cudaSuccess ? SF_OK : cuda_fail(c, e, "ratio launch");
}
}  // namespace

sf_status sf_weighted_filter(sf_ctx *c, const float *d_cube, const float *d_weights, int32_t filter, int32_t den,
                             float *d_out, void *stream)
{
    sf_status s = weighted_check(c, d_cube, d_weights, den);
    if (s != SF_OK) return s;
    if (filter < 0 || filter >= (int)c->filt.size()) return fail(c, SF_EINVAL, "filter index %d", filter);
    if (!d_out || !aligned16(d_out)) return fail(c, SF_EINVAL, "d_out must be a 16-byte aligned buffer");
    DeviceGuard dg(c->device);
    if ((s = weighted_scratch(c, den)) != SF_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    float *p = c->wscratch;
    const cudaError_t e = sf_launch_w_product(d_cube, d_weights, p, c->nvox, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "product launch");
    return weighted_one(c, p, d_weights, filter, den, d_out, st);
}

sf_status sf_weighted_detect(sf_ctx *c, const float *d_cube, const float *d_weights, int32_t den, uint32_t *d_mask,
                             float *d_mean, float *d_std, void *stream)
{
    sf_status s = weighted_check(c, d_cube, d_weights, den);
    if (s != SF_OK) return s;
    if (!d_mask) return fail(c, SF_EINVAL, "NULL mask");
    if ((d_mean == nullptr) != (d_std == nullptr))
        return fail(c, SF_EINVAL, "d_mean and d_std must both be NULL or both be set");
    DeviceGuard dg(c->device);
    if ((s = weighted_scratch(c, den)) != SF_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cube = align_up((size_t)c->nvox * sizeof(float), 256) / sizeof(float);
    float *p = c->wscratch, *num = c->wscratch + cube;
    cudaError_t e = sf_launch_w_product(d_cube, d_weights, p, c->nvox, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "product launch");
    if (c->fused && (s = weighted_plan(c, den)) != SF_OK) return s;
    const sf_ctx::WPlan &W = c->wplan[den];
    if (c->fused && W.ready && (den == 1 || (s = weighted_gauss_twin(c)) == SF_OK)) {
        /* fused: x passes of d*w (this context's scratch) and of w (the
         * twin's), then one window kernel over (denominator, numerator)
         * pairs that divides before the moments */
        sf_ctx *tw = den == 1 ? c->boxtwin : c->gausstwin;
        for (size_t i = 0; i < c->xlaunch.size(); ++i)
            if ((s = run_xpass(c, c->xlaunch[i], c->xgroups[i], p, st)) != SF_OK) return s;
        for (size_t i = 0; i < tw->xlaunch.size(); ++i)
            if ((s = run_xpass(tw, tw->xlaunch[i], tw->xgroups[i], d_weights, st)) != SF_OK)
                return fail(c, s, "%s", tw->err.c_str());
        sf_dargs da{};
        sf_ctx::WPlan &Wm = c->wplan[den];
        for (size_t i = 0; i < W.srcs.size(); ++i) {
            const DetectSource &d = W.srcs[i];
            const void *src = d.den ? (d.slot < 0 ? (const void *)d_weights
                                                  : (const void *)((const char *)tw->scratch + (size_t)d.slot * tw->cube_bytes))
                                    : (d.slot < 0 ? (const void *)p
                                                  : (const void *)((const char *)c->scratch + (size_t)d.slot * c->cube_bytes));
            da.src[i] = src;
            for (size_t q = 0; q < d.filters.size(); ++q) da.fidx[i][q] = d.filters[q];
            if (W.tma && !encode_map_dims(c, src, c->cfg.nx, c->cfg.ny, c->cfg.nz, c->dSROW, d.ry, &Wm.maps[i]))
                return fail(c, SF_ECUDA, "tensor map encoding failed");
        }
        da.mask = d_mask;
        da.mean = d_mean;
        da.stdv = d_std;
        da.nx = c->cfg.nx;
        da.ny = c->cfg.ny;
        da.nz = c->cfg.nz;
        da.nw32 = c->nw32;
        da.nwx = c->nwx;
        da.nwy = c->nwy;
        da.nwz = c->nwz;
        da.nwin = c->nwin;
        da.k = c->cfg.k;
        da.err = c->err_flag;
        da.wait_ns = c->wait_ns;
        da.wid0 = 0;
        void *args[] = {&da, (void *)W.taps.data(), (void *)Wm.maps.data()};
        return launch(c, W.L, args, st, "weighted window kernel launch");
    }
    if (s != SF_OK) return s;
    for (int f = 0; f < (int)c->filt.size(); ++f) {
        /* the ratio overwrites the numerator in place */
        if ((s = weighted_one(c, p, d_weights, f, den, num, st)) != SF_OK) return s;
        float *m = d_mean ? d_mean + (size_t)f * c->nwin : c->wstats;
        float *sd = d_std ? d_std + (size_t)f * c->nwin : c->wstats + c->nwin;
        if ((s = sf_stats(c, num, m, sd, stream)) != SF_OK) return s;
        if ((s = sf_threshold(c, num, m, sd, d_mask, f > 0 ? 1 : 0, stream)) != SF_OK) return s;
    }
    return SF_OK;
}

sf_status sf_synchronize(sf_ctx *c, void *stream)
{
    sf_status s = check_live(c, true);
    if (s != SF_OK) return s;
    if (c->sectioned) {
        for (sf_ctx *u : c->sub)
            if (u && (s = sf_synchronize(u, stream)) != SF_OK) return fail(c, s, "section: %s", u->err.c_str());
        return SF_OK;
    }
    DeviceGuard dg(c->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronise");
    int flag = 0;
    if ((e = cudaMemcpy(&flag, c->err_flag, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(c, e, "error flag read");
    if (flag) {
        cudaMemset(c->err_flag, 0, sizeof(int));
        return fail(c, SF_ETIMEOUT, "a kernel's bounded wait (shared-memory loads, or another CTA's "
                                    "x pass) expired (flag 0x%x)", (unsigned)flag);
    }
    return SF_OK;
}

sf_status sf_set_wait_limit(sf_ctx *c, int64_t limit_ns)
{
    sf_status s = check_live(c, true);
    if (s != SF_OK) return s;
    if (limit_ns < 1000 || limit_ns > 60000000000LL)
        return fail(c, SF_EINVAL, "wait limit %lld ns outside [1 us, 60 s]", (long long)limit_ns);
    c->wait_ns = limit_ns;
    if (c->sectioned) {
        for (sf_ctx *u : c->sub)
            if (u && (s = sf_set_wait_limit(u, limit_ns)) != SF_OK) return fail(c, s, "section: %s", u->err.c_str());
        return SF_OK;
    }
    /* the persistent graph holds its launch arguments: capture it again */
    if (c->pready) {
        DeviceGuard dg(c->device);
        if (c->gpending) {
            cudaError_t e = cudaEventSynchronize(c->gdone);
            if (e != cudaSuccess) return cuda_fail(c, e, "previous batch");
            c->gpending = false;
        }
        return plan_persist(c, sf_ctx::PersistPlan(c->pp));
    }
    return SF_OK;
}

sf_status sf_test_stall_batch(sf_ctx *c, int32_t extra)
{
    sf_status s = check_live(c);
    if (s != SF_OK) return s;
    if (!c->batch) return fail(c, SF_EINVAL, "the stall hook takes a batched context");
    if (extra < 0 || extra > 1000000) return fail(c, SF_EINVAL, "extra %d outside [0, 1e6]", (int)extra);
    if (c->xy_sigma.empty()) return fail(c, SF_EINVAL, "the bank has no x pass to wait for");
    DeviceGuard dg(c->device);
    if (c->gpending) {
        cudaError_t e = cudaEventSynchronize(c->gdone);
        if (e != cudaSuccess) return cuda_fail(c, e, "previous batch");
        c->gpending = false;
    }
    c->stall_extra = extra;
    sf_ctx::PersistPlan q;   /* x items inside the persistent kernel, whole cubes */
    q.xbatch = false;
    return plan_persist(c, q);
}

}  /* extern "C" */
