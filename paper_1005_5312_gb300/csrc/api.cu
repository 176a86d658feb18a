// C ABI of the START library (declared in include/start.h): context
// lifetime, input staging (host or device pointers), validation, the
// build / state / solve / ionise sequence and test introspection.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"

namespace st {


// ---------------------------------------------------------------- buffers and errors
// Device buffers come from a library-owned, stream-ordered memory pool (one
// per device, memory kept reserved after a free): growing a buffer never
// synchronises the device, so contexts on different streams -- concurrent
// requests of a server -- do not stall each other.  Allocations and frees
// are ordered on the stream of the context being served (thread-local,
// set on entry to every public call).
namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};
std::atomic<long long> g_bytes{0};
thread_local cudaStream_t tl_stream = nullptr;

cudaMemPool_t device_pool()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = pool;
    }
    return g_pool[dev];
}
}  // namespace

void set_thread_stream(cudaStream_t s) { tl_stream = s; }
cudaStream_t thread_stream() { return tl_stream; }

int ensure(DBuf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (bytes <= b.cap) return START_OK;
    release(b);
    size_t want = bytes + bytes / 8 + 256;
    cudaMemPool_t pool = device_pool();
    void *p = nullptr;
    if (!pool || cudaMallocFromPoolAsync(&p, want, pool, tl_stream) != cudaSuccess) {
        cudaGetLastError();
        return START_ENOMEM;
    }
    b.p = p;
    b.cap = want;
    g_bytes += (long long)want;
    return START_OK;
}

int ensure_keep(DBuf &b, size_t bytes, size_t used, cudaStream_t s)
{
    if (bytes <= b.cap) return START_OK;
    cudaMemPool_t pool = device_pool();
    void *q = nullptr;
    if (!pool || cudaMallocFromPoolAsync(&q, bytes, pool, s) != cudaSuccess) {
        cudaGetLastError();
        return START_ENOMEM;
    }
    if (b.p && used) cudaMemcpyAsync(q, b.p, std::min(used, b.cap), cudaMemcpyDeviceToDevice, s);
    if (b.p) {
        cudaFreeAsync(b.p, s);
        g_bytes -= (long long)b.cap;
    }
    b.p = q;
    b.cap = bytes;
    g_bytes += (long long)bytes;
    return START_OK;
}

void release(DBuf &b)
{
    if (b.p) {
        cudaFreeAsync(b.p, tl_stream);
        g_bytes -= (long long)b.cap;
    }
    b.p = nullptr;
    b.cap = 0;
}

long long bytes_in_use() { return g_bytes.load(); }

void phase_mark(start_ctx *c, int phase, bool end)
{
    if (!c->p.timing) return;
    std::vector<cudaEvent_t> &v = c->pev[phase];
    const size_t k = 2 * (size_t)c->pcount[phase] + (end ? 1 : 0);
    while (v.size() <= k) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        v.push_back(e);
    }
    cudaEventRecord(v[k], c->stream);
    if (end) ++c->pcount[phase];
}

int set_err(start_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}

int cuda_check(start_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return START_OK;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return set_err(c, START_ECUDA, m);
}

static bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Copies n bytes of a caller pointer (host or device) into b.
static int stage_in(start_ctx *c, DBuf &b, const void *src, size_t n)
{
    ST_TRY(ensure(b, n));
    if (n) ST_CUDA(c, cudaMemcpyAsync(b.p, src, n, cudaMemcpyDefault, c->stream));
    return START_OK;
}

// Copies n bytes of device data to a caller pointer (host or device);
// synchronises when the destination is host memory.
static int copy_out(start_ctx *c, void *dst, const void *src, size_t n)
{
    if (!n || !dst) return START_OK;
    ST_CUDA(c, cudaMemcpyAsync(dst, src, n, cudaMemcpyDefault, c->stream));
    if (!is_device_ptr(dst)) ST_CUDA(c, cudaStreamSynchronize(c->stream));
    return START_OK;
}

// Makes the context's device current and its stream the thread's allocation
// stream for the duration of a public call; restores both on exit.
struct DeviceGuard {
    int prev = -1;
    cudaStream_t prev_stream = nullptr;
    explicit DeviceGuard(const start_ctx *c)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        if (prev != c->device) cudaSetDevice(c->device);
        prev_stream = thread_stream();
        set_thread_stream(c->stream);
    }
    ~DeviceGuard()
    {
        set_thread_stream(prev_stream);
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// ---------------------------------------------------------------- small kernels
__global__ void k_check_pos_h(const float *h, long long n, unsigned long long *bad)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(isfinite(h[i]) && h[i] > 0.f)) atomicAdd(bad, 1ull);
}
__global__ void k_check_nonneg_f(const float *v, long long n, unsigned long long *bad)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(isfinite(v[i]) && v[i] >= 0.f)) atomicAdd(bad, 1ull);
}
__global__ void k_check_nonneg_d(const double *v, long long n, unsigned long long *bad, int strict)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(isfinite(v[i]) && (strict ? v[i] > 0.0 : v[i] >= 0.0))) atomicAdd(bad, 1ull);
}
__global__ void k_check_unit_d(const double *v, long long n, unsigned long long *bad)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(v[i] >= 0.0 && v[i] <= 1.0)) atomicAdd(bad, 1ull);
}

__global__ void k_fill_d(double *v, long long n, double x)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = x;
}

__global__ void k_scatter_d(const double *in, const u32 *inv, long long n, double *out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[inv[i]] = in[i];
}

__global__ void k_invert(const u32 *perm, long long n, u32 *inv)
{
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) inv[perm[r]] = (u32)r;
}

// Morton-ordered particle records from the staged SoA inputs.
__global__ void k_gather_particles(const float *pos, const float *h, const double *V,
                                   const u32 *perm, long long n, float4 *pq, float *ph,
                                   double *Vm, float *nH, double *y, float *gam)
{
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    u32 i = perm[r];
    pq[r] = make_float4(pos[i], pos[n + i], pos[2 * n + i], 0.f);
    ph[r] = h[i];
    if (V) Vm[r] = V[i];
    else Vm[r] = 0.0;
    nH[r] = 0.f;
    y[r] = 1.0;
    gam[r] = 0.f;
}

__global__ void k_gather_sources(const float *pos, const double *L, const u32 *perm, long long n,
                                 double L_unit, float4 *sq, double *sL)
{
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    u32 i = perm[r];
    double Lj = L[i];
    sq[r] = make_float4(pos[i], pos[n + i], pos[2 * n + i],
                        __double2float_rn(__ddiv_rn(Lj, L_unit)));
    sL[r] = Lj;
}

__global__ void k_set_state(const float *nH_in, const double *y_in, const u32 *inv, long long n,
                            float *nH, double *y, float4 *pq)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    u32 r = inv[i];
    double yy = y_in ? y_in[i] : 1.0;
    float nh = nH_in[i];
    nH[r] = nh;
    y[r] = yy;
    pq[r].w = __double2float_rn(yy * (double)nh);
}

__global__ void k_set_nHI(const float *nHI, const u32 *inv, long long n, float4 *pq)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pq[inv[i]].w = nHI[i];
}

template <class T>
__global__ void k_to_input_order(const T *m, const u32 *perm, long long n, T *out)
{
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) out[perm[r]] = m[r];
}

static unsigned long long read_counter(start_ctx *c, int slot)
{
    unsigned long long v = 0;
    cudaMemcpyAsync(&v, c->counters.as<unsigned long long>() + slot, sizeof(v),
                    cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    return v;
}

static int check_bad(start_ctx *c, const char *what)
{
    unsigned long long bad = read_counter(c, C_BAD_INPUT);
    ST_CUDA(c, cudaGetLastError());
    if (bad) {
        ST_CUDA(c, cudaMemsetAsync(c->counters.as<unsigned long long>() + C_BAD_INPUT, 0,
                                   sizeof(unsigned long long), c->stream));
        return set_err(c, START_EINVAL, std::string("invalid values in ") + what);
    }
    return START_OK;
}

// Reorders Morton-row CSR (u32 or u64 offsets) into input order on the host.
template <class O>
static void csr_to_input(long long n, const std::vector<O> &moff, const std::vector<u32> &mval,
                         const std::vector<u32> &porig, bool map_vals, std::vector<u64> &off,
                         std::vector<u32> &val)
{
    std::vector<u64> cnt(n + 1, 0);
    for (long long r = 0; r < n; ++r) cnt[porig[r]] = (u64)(moff[r + 1] - moff[r]);
    off.assign(n + 1, 0);
    for (long long i = 0; i < n; ++i) off[i + 1] = off[i] + cnt[i];
    val.resize(off[n]);
    for (long long r = 0; r < n; ++r) {
        u64 w = off[porig[r]];
        for (O e = moff[r]; e < moff[r + 1]; ++e) val[w++] = map_vals ? porig[mval[e]] : mval[e];
    }
}

// ---------------------------------------------------------------- batches
// Merging one problem's structures into a batch's forest: plain copies, and
// index arrays shifted by the problem's offsets (kNone kept).
__global__ void k_shift_u32(const u32 *in, long long n, u32 add, u32 *out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i] == 0xffffffffu ? 0xffffffffu : in[i] + add;   // "none" kept
}

__global__ void k_shift_meta(const uint4 *in, long long n, u32 node0, u32 memb0, uint4 *out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        uint4 m = in[i];
        out[i] = make_uint4(m.x + node0, m.y + memb0, m.z, m.w);
    }
}

__global__ void k_fill_range(uint2 *tr, float *rf2, long long n, uint2 r, float f)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        tr[i] = r;
        rf2[i] = f;
    }
}

extern "C" int start_destroy(start_ctx *c);

int destroy_batch_parts(start_ctx *c)
{
    for (start_ctx *b : c->bsub) start_destroy(b);
    c->bsub.clear();
    return START_OK;
}

static int copy_dev(start_ctx *c, void *dst, const void *src, size_t bytes)
{
    if (!bytes) return START_OK;
    return cuda_check(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream),
                      "batch copy");
}

static int shift_copy(start_ctx *c, u32 *dst, const u32 *src, long long n, u32 add)
{
    if (n <= 0) return START_OK;
    k_shift_u32<<<grid_for(n, 256), 256, 0, c->stream>>>(src, n, add, dst);
    ++c->launches;
    return cuda_check(c, cudaGetLastError(), "k_shift_u32");
}

static void release_all(start_ctx *c)
{
    c->rb_n = c->rb_geo_n = 0;
    destroy_batch_parts(c);
    resident_reset(c);
    if (c->r_cap) cudaStreamDestroy(c->r_cap);
    c->r_cap = nullptr;
    DBuf *all[] = {&c->pq, &c->ph, &c->porig, &c->pinv, &c->pkey, &c->nH, &c->mass_in,
                   &c->mass_s, &c->h2_in, &c->w_save, &c->heat, &c->spec_tab, &c->y, &c->V,
                   &c->gam, &c->eL, &c->eLs, &c->sq, &c->sorig, &c->skey, &c->sL,
                   &c->nb_off, &c->nb_idx, &c->lcount, &c->loff, &c->pent, &c->ptgt,
                   &c->pcon, &c->tk[0], &c->tk[1], &c->tv[0], &c->tv[1], &c->hist,
                   &c->scan_tmp, &c->stage, &c->flags, &c->counters, &c->m_vid, &c->m_j, &c->m_ord, &c->pord, &c->m_nx0, &c->m_dl,
                   &c->r_j, &c->r_up, &c->r_dl, &c->r_next, &c->r_tau, &c->r_pos, &c->r_lvl, &c->r_vid,
                   &c->m_st[0], &c->m_st[1], &c->m_ups, &c->m_fr, &c->m_hard, &c->m_part, &c->m_table,
                   &c->w_scratch, &c->w_over, &c->ctr_save, &c->g_hist, &c->gacc, &c->klum_big, &c->trange, &c->trf2,
                   &c->rb_mask, &c->rb_geo, &c->rb_amax, &c->m_w[0], &c->m_w[1]};
    for (DBuf *b : all) release(*b);
    tree_release(c->pt);
    tree_release(c->stree);
    tree_release(c->et);
    for (int k = 0; k < START_NPHASES; ++k) {
        for (cudaEvent_t e : c->pev[k]) cudaEventDestroy(e);
        c->pev[k].clear();
        c->pcount[k] = 0;
    }
    for (int k = 0; k < 4; ++k)
        if (c->hev[k]) cudaEventDestroy(c->hev[k]);
    for (cudaEvent_t &e : c->lev_ev)
        if (e) cudaEventDestroy(e);
}

}  // namespace st

using namespace st;

// ---------------------------------------------------------------- staging buffers
namespace {
struct Staged {
    DBuf pos, h, spos, L, V;
    ~Staged()
    {
        release(pos);
        release(h);
        release(spos);
        release(L);
        release(V);
    }
};
}  // namespace

extern "C" {

int start_default_params(start_params *p)
{
    if (!p) return START_EINVAL;
    memset(p, 0, sizeof(*p));
    p->src_leaf = 1;
    p->ptree_leaf = 16;
    p->march_group = 2;
    p->march_mode = 1;
    p->row_warps = 8;
    p->walk_warp = 0;
    p->row_bins = 4;
    p->sigma_cm2 = 6.3e-18;
    p->len_unit_cm = 3.0857e21;
    p->L_unit = 1e48;
    p->alpha_A = 4.18e-13;
    p->alpha_B = 2.59e-13;
    p->tau_cut = 110.0;
    p->hop_cap = 0;
    p->spin_cap = 1 << 24;
    p->stream = nullptr;
    return START_OK;
}

static int check_params(start_params &d)
{
    if (d.src_leaf < 1 || d.ptree_leaf < 1 || !(d.sigma_cm2 > 0) || !(d.len_unit_cm > 0) ||
        !(d.L_unit > 0) || !(d.alpha_A >= 0) || !(d.alpha_B >= 0) || !(d.tau_cut > 0))
        return START_EINVAL;
    if (d.march_group != 0 && d.march_group != 1 && d.march_group != 2 && d.march_group != 4 &&
        d.march_group != 8 && d.march_group != 16 && d.march_group != 32)
        return START_EINVAL;
    if (d.march_group == 0) d.march_group = 2;
    if (d.march_mode != 0 && d.march_mode != 1) return START_EINVAL;
    if (d.row_warps != 0 && d.row_warps != 4 && d.row_warps != 8) return START_EINVAL;
    if (d.thermal != 0 && d.thermal != 1) return START_EINVAL;
    if (d.lum_kernel != 0 && d.lum_kernel != 1) return START_EINVAL;
    if (d.walk_warp != 0 && d.walk_warp != 1) return START_EINVAL;
    if (d.row_bins != 0 && (d.row_bins < 2 || d.row_bins > 6)) return START_EINVAL;
    if (d.link_counts != 0 && d.link_counts != 1) return START_EINVAL;
    if (d.row_warps == 0) d.row_warps = 8;
    if (d.max_pairs < 0 || d.hop_cap < 0) return START_EINVAL;
    if (!(d.T_eff == 0.0 || (d.T_eff >= 500.0 && d.T_eff <= 1e7))) return START_EINVAL;
    if (!(d.T_rec == 0.0 || (d.T_rec >= 100.0 && d.T_rec <= 1e5))) return START_EINVAL;
    return START_OK;
}

int start_create(start_ctx **out, const start_params *p)
{
    if (!out) return START_EINVAL;
    *out = nullptr;
    start_params d;
    start_default_params(&d);
    if (p) d = *p;
    if (check_params(d) != START_OK) return START_EINVAL;
    start_ctx *c = new (std::nothrow) start_ctx();
    if (!c) return START_ENOMEM;
    c->p = d;
    c->stream = (cudaStream_t)d.stream;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return START_ECUDA;
    }
    DeviceGuard g(c);
    if (ensure(c->counters, C_COUNT * sizeof(unsigned long long)) ||
        cudaMemsetAsync(c->counters.p, 0, C_COUNT * sizeof(unsigned long long), c->stream) !=
            cudaSuccess) {
        cudaGetLastError();
        release_all(c);
        delete c;
        return START_ENOMEM;
    }
    *out = c;
    return START_OK;
}

int start_set_params(start_ctx *c, const start_params *p)
{
    if (!c || !p) return START_EINVAL;
    start_params d = *p;
    if (check_params(d) != START_OK) return set_err(c, START_EINVAL, "invalid parameters");
    DeviceGuard g(c);
    if ((cudaStream_t)d.stream != c->stream) {
        cudaStreamSynchronize(c->stream);
        resident_reset(c);   // the captured graph belongs to the old stream's sequence
    }
    if (d.reuse_chains != c->p.reuse_chains || d.sigma_cm2 != c->p.sigma_cm2 ||
        d.len_unit_cm != c->p.len_unit_cm || d.L_unit != c->p.L_unit || d.T_eff != c->p.T_eff)
        resident_reset(c);
    c->p = d;
    c->stream = (cudaStream_t)d.stream;
    return START_OK;
}

int start_destroy(start_ctx *c)
{
    if (!c) return START_EINVAL;
    DeviceGuard g(c);
    cudaStreamSynchronize(c->stream);
    release_all(c);
    cudaStreamSynchronize(c->stream);
    delete c;
    return START_OK;
}

int start_build_trees(start_ctx *c, const float *pos, const float *h, long long n_p,
                      const float *src_pos, const double *src_L, long long n_s, const double *V,
                      unsigned flags)
{
    if (!c) return START_EINVAL;
    DeviceGuard g(c);
    c->built = c->has_state = c->solved = false;
    c->nbatch = 0;
    c->rb_n = 0;
    resident_reset(c);
    if (n_p < 0 || n_s < 0) return set_err(c, START_EINVAL, "negative size");
    if (n_p >= START_MAX_N || n_s >= START_MAX_N)
        return set_err(c, START_ERANGE, "n_p and n_s must be below 2^30");
    if ((n_p && (!pos || !h)) || (n_s && (!src_pos || !src_L)))
        return set_err(c, START_EINVAL, "NULL input array");
    bool diffuse = (flags & START_DIFFUSE) != 0;
    if (diffuse && n_p && !V) return set_err(c, START_EINVAL, "diffuse mode needs V");
    c->np = n_p;
    c->ns = n_s;
    c->diffuse = diffuse;
    cudaStream_t s = c->stream;
    unsigned long long *ctr = c->counters.as<unsigned long long>();
    ST_CUDA(c, cudaMemsetAsync(ctr, 0, C_COUNT * sizeof(unsigned long long), s));

    phase_mark(c, START_PHASE_BUILD, false);
    Staged in;
    ST_TRY(stage_in(c, in.pos, pos, 3 * n_p * sizeof(float)));
    ST_TRY(stage_in(c, in.h, h, n_p * sizeof(float)));
    ST_TRY(stage_in(c, in.spos, src_pos, 3 * n_s * sizeof(float)));
    ST_TRY(stage_in(c, in.L, src_L, n_s * sizeof(double)));
    if (diffuse) ST_TRY(stage_in(c, in.V, V, n_p * sizeof(double)));
    ST_CUDA(c, cudaMemsetAsync(ctr + C_INTERNAL, 0, sizeof(unsigned long long), s));
    if (n_p) { k_check_pos_h<<<grid_for(n_p, 256), 256, 0, s>>>(in.h.as<float>(), n_p, ctr + C_BAD_INPUT); ++c->launches; }
    if (n_s) { k_check_nonneg_d<<<grid_for(n_s, 256), 256, 0, s>>>(in.L.as<double>(), n_s, ctr + C_BAD_INPUT, 0); ++c->launches; }
    if (diffuse && n_p)
        k_check_nonneg_d<<<grid_for(n_p, 256), 256, 0, s>>>(in.V.as<double>(), n_p, ctr + C_BAD_INPUT, 1); ++c->launches;
    ST_TRY(check_bad(c, "h, src_L or V"));
    if (n_p + n_s == 0) {
        c->pt.n = c->stree.n = c->et.n = 0;
        c->nb_total = 0;
        c->built = true;
        return START_OK;
    }
    ST_TRY(compute_frame(c, in.pos.as<float>(), n_p, in.spos.as<float>(), n_s, &c->fr));

    // particles: keys, stable sort, Morton-ordered records
    size_t P = (size_t)(n_p ? n_p : 1), S = (size_t)(n_s ? n_s : 1);
    if (ensure(c->pkey, P * 8) || ensure(c->tk[1], P * 8) || ensure(c->porig, P * 4) ||
        ensure(c->pinv, P * 4) || ensure(c->pq, P * 16) || ensure(c->ph, P * 4) ||
        ensure(c->nH, P * 4) || ensure(c->y, P * 8) || ensure(c->V, P * 8) || ensure(c->Tg, P * 8) ||
        ensure(c->gam, P * 4) || ensure(c->eL, P * 8) || ensure(c->eLs, P * 4) ||
        ensure(c->skey, S * 8) || ensure(c->tv[1], S * 8) || ensure(c->sorig, S * 4) ||
        ensure(c->sq, S * 16) || ensure(c->sL, S * 8))
        return set_err(c, START_ENOMEM, "out of device memory (inputs)");
    u64 *pks = c->tk[1].as<u64>();
    if (n_p) {
        ST_TRY(morton_keys(c, in.pos.as<float>(), n_p, c->fr, pks, c->porig.as<u32>()));
        ST_CUDA(c, cudaMemcpyAsync(c->pkey.p, pks, n_p * 8, cudaMemcpyDeviceToDevice, s));
        ST_TRY(radix_sort_pairs(c, pks, c->porig.as<u32>(), n_p));
        k_invert<<<grid_for(n_p, 256), 256, 0, s>>>(c->porig.as<u32>(), n_p, c->pinv.as<u32>()); ++c->launches;
        k_gather_particles<<<grid_for(n_p, 256), 256, 0, s>>>(
            in.pos.as<float>(), in.h.as<float>(), diffuse ? in.V.as<double>() : nullptr,
            c->porig.as<u32>(), n_p, c->pq.as<float4>(), c->ph.as<float>(), c->V.as<double>(),
            c->nH.as<float>(), c->y.as<double>(), c->gam.as<float>()); ++c->launches;
        ST_CUDA(c, cudaMemsetAsync(c->eL.p, 0, n_p * 8, s));
        ST_CUDA(c, cudaMemsetAsync(c->eLs.p, 0, n_p * 4, s));
        k_fill_d<<<grid_for(n_p, 256), 256, 0, s>>>(c->Tg.as<double>(), n_p, 1e4); ++c->launches;
        ST_CUDA(c, cudaGetLastError());
    }
    u64 *sks = c->tv[1].as<u64>();
    if (n_s) {
        ST_TRY(morton_keys(c, in.spos.as<float>(), n_s, c->fr, sks, c->sorig.as<u32>()));
        ST_CUDA(c, cudaMemcpyAsync(c->skey.p, sks, n_s * 8, cudaMemcpyDeviceToDevice, s));
        ST_TRY(radix_sort_pairs(c, sks, c->sorig.as<u32>(), n_s));
        k_gather_sources<<<grid_for(n_s, 256), 256, 0, s>>>(in.spos.as<float>(), in.L.as<double>(),
                                                            c->sorig.as<u32>(), n_s, c->p.L_unit,
                                                            c->sq.as<float4>(), c->sL.as<double>()); ++c->launches;
        ST_CUDA(c, cudaGetLastError());
    }
    ST_TRY(build_octree(c, c->pt, pks, n_p, c->p.ptree_leaf, c->fr));
    ST_TRY(build_octree(c, c->stree, sks, n_s, c->p.src_leaf, c->fr));
    ST_TRY(tree_moments(c, c->stree, c->sq.as<float4>(), c->sL.as<double>(), c->p.L_unit));
    if (diffuse) ST_TRY(build_octree(c, c->et, pks, n_p, c->p.src_leaf, c->fr));
    else c->et.n = 0;
    ST_TRY(build_neighbours(c));
    phase_mark(c, START_PHASE_BUILD, true);
    ST_CUDA(c, cudaStreamSynchronize(s));
    ST_CUDA(c, cudaGetLastError());
    if (read_counter(c, C_INTERNAL)) return set_err(c, START_ECUDA, "internal inconsistency (trees or neighbour lists)");
    c->built = true;
    return START_OK;
}

int start_build_batch(start_ctx *c, int nb, const long long *n_p, const long long *n_s,
                                 const float *const *pos, const float *const *h,
                                 const float *const *src_pos, const double *const *src_L)
{
    if (!c) return START_EINVAL;
    DeviceGuard g(c);
    c->built = c->has_state = c->solved = false;
    c->nbatch = 0;
    c->rb_n = 0;
    resident_reset(c);
    if (nb < 1 || !n_p || !n_s || !pos || !h || !src_pos || !src_L)
        return set_err(c, START_EINVAL, "a batch needs n >= 1 problems and their arrays");
    long long P = 0, S = 0;
    for (int b = 0; b < nb; ++b) {
        if (n_p[b] < 0 || n_s[b] < 0) return set_err(c, START_EINVAL, "negative size");
        P += n_p[b];
        S += n_s[b];
    }
    if (P >= START_MAX_N || S >= START_MAX_N)
        return set_err(c, START_ERANGE, "a batch holds below 2^30 particles and sources");
    // every problem built on its own (its frame, trees and neighbour lists), in
    // contexts that share this one's stream and parameters
    while ((int)c->bsub.size() < nb) {
        start_ctx *b = nullptr;
        start_params q = c->p;
        q.timing = 0;
        int rc = start_create(&b, &q);
        if (rc != START_OK) return set_err(c, rc, "batch: creating a part");
        c->bsub.push_back(b);
    }
    long long N = 0, NB = 0;
    float cmag = 0.f;
    for (int b = 0; b < nb; ++b) {
        start_ctx *q = c->bsub[b];
        q->p = c->p;
        q->p.timing = 0;
        q->stream = c->stream;
        int rc = start_build_trees(q, pos[b], h[b], n_p[b], src_pos[b], src_L[b], n_s[b], nullptr,
                                   0u);
        if (rc != START_OK) return set_err(c, rc, "batch part " + std::to_string(b) + ": " + q->err);
        N += q->stree.n;
        NB += q->nb_total;
        if (q->np + q->ns > 0 && q->fr.cmag > cmag) cmag = q->fr.cmag;
        c->launches += q->launches;
        q->launches = 0;
    }
    if (N >= (1LL << 31)) return set_err(c, START_ERANGE, "a batch's forest is too large");
    size_t Pz = (size_t)(P ? P : 1), Sz = (size_t)(S ? S : 1), Nz = (size_t)(N ? N : 1);
    Tree &t = c->stree;
    if (ensure(c->pq, Pz * 16) || ensure(c->ph, Pz * 4) || ensure(c->porig, Pz * 4) ||
        ensure(c->pinv, Pz * 4) || ensure(c->pkey, Pz * 8) || ensure(c->nH, Pz * 4) ||
        ensure(c->y, Pz * 8) || ensure(c->V, Pz * 8) || ensure(c->Tg, Pz * 8) ||
        ensure(c->gam, Pz * 4) || ensure(c->eL, Pz * 8) || ensure(c->eLs, Pz * 4) ||
        ensure(c->nb_off, (Pz + 1) * 4) || ensure(c->nb_idx, (size_t)(NB ? NB : 1) * 4) ||
        ensure(c->sq, Sz * 16) || ensure(c->sL, Sz * 8) || ensure(c->sorig, Sz * 4) ||
        ensure(c->skey, Sz * 8) || ensure(t.box, Nz * 16) || ensure(t.meta, Nz * 16) ||
        ensure(t.cube, Nz * 32) || ensure(t.level, Nz * 4) || ensure(t.parent, Nz * 4) ||
        ensure(t.leafof, Sz * 4) || ensure(t.vsrc, Nz * 16) || ensure(t.L, Nz * 8) ||
        ensure(t.M, Nz * 24) || ensure(c->trange, Pz * 8) || ensure(c->trf2, Pz * 4))
        return set_err(c, START_ENOMEM, "out of device memory (batch)");
    long long p0 = 0, s0 = 0, n0 = 0, e0 = 0;
    for (int b = 0; b < nb; ++b) {
        start_ctx *q = c->bsub[b];
        const long long np = q->np, ns = q->ns, nn = q->stree.n, ne = q->nb_total;
        if (np) {
            ST_TRY(copy_dev(c, c->pq.as<float4>() + p0, q->pq.p, np * 16));
            ST_TRY(copy_dev(c, c->ph.as<float>() + p0, q->ph.p, np * 4));
            ST_TRY(copy_dev(c, c->pkey.as<u64>() + p0, q->pkey.p, np * 8));
            ST_TRY(copy_dev(c, c->V.as<double>() + p0, q->V.p, np * 8));
            ST_TRY(copy_dev(c, c->nH.as<float>() + p0, q->nH.p, np * 4));
            ST_TRY(copy_dev(c, c->y.as<double>() + p0, q->y.p, np * 8));
            ST_TRY(copy_dev(c, c->gam.as<float>() + p0, q->gam.p, np * 4));
            ST_TRY(copy_dev(c, c->Tg.as<double>() + p0, q->Tg.p, np * 8));
            ST_TRY(shift_copy(c, c->porig.as<u32>() + p0, q->porig.as<u32>(), np, (u32)p0));
            ST_TRY(shift_copy(c, c->pinv.as<u32>() + p0, q->pinv.as<u32>(), np, (u32)p0));
            ST_TRY(shift_copy(c, c->nb_off.as<u32>() + p0, q->nb_off.as<u32>(), np, (u32)e0));
            ST_TRY(shift_copy(c, c->nb_idx.as<u32>() + e0, q->nb_idx.as<u32>(), ne, (u32)p0));
            const double rf = 1e-6 * q->fr.side;
            k_fill_range<<<grid_for(np, 256), 256, 0, c->stream>>>(
                c->trange.as<uint2>() + p0, c->trf2.as<float>() + p0, np,
                make_uint2((u32)n0, (u32)(n0 + nn)), (float)(rf * rf));
            ++c->launches;
        }
        if (ns) {
            ST_TRY(copy_dev(c, c->sq.as<float4>() + s0, q->sq.p, ns * 16));
            ST_TRY(copy_dev(c, c->sL.as<double>() + s0, q->sL.p, ns * 8));
            ST_TRY(copy_dev(c, c->skey.as<u64>() + s0, q->skey.p, ns * 8));
            ST_TRY(shift_copy(c, c->sorig.as<u32>() + s0, q->sorig.as<u32>(), ns, (u32)s0));
            ST_TRY(shift_copy(c, t.leafof.as<u32>() + s0, q->stree.leafof.as<u32>(), ns, (u32)n0));
        }
        if (nn) {
            const Tree &u = q->stree;
            ST_TRY(copy_dev(c, t.box.as<float4>() + n0, u.box.p, nn * 16));
            ST_TRY(copy_dev(c, t.cube.as<double>() + 4 * n0, u.cube.p, nn * 32));
            ST_TRY(copy_dev(c, t.level.as<int>() + n0, u.level.p, nn * 4));
            ST_TRY(copy_dev(c, t.vsrc.as<float4>() + n0, u.vsrc.p, nn * 16));
            ST_TRY(copy_dev(c, t.L.as<double>() + n0, u.L.p, nn * 8));
            ST_TRY(copy_dev(c, t.M.as<double>() + 3 * n0, u.M.p, nn * 24));
            ST_TRY(shift_copy(c, t.parent.as<u32>() + n0, u.parent.as<u32>(), nn, (u32)n0));
            k_shift_meta<<<grid_for(nn, 256), 256, 0, c->stream>>>(
                u.meta.as<uint4>(), nn, (u32)n0, (u32)s0, t.meta.as<uint4>() + n0);
            ++c->launches;
        }
        p0 += np;
        s0 += ns;
        n0 += nn;
        e0 += ne;
    }
    u32 etot = (u32)NB;
    ST_CUDA(c, cudaMemcpyAsync(c->nb_off.as<u32>() + P, &etot, 4, cudaMemcpyHostToDevice,
                               c->stream));
    if (P) {
        ST_CUDA(c, cudaMemsetAsync(c->eL.p, 0, P * 8, c->stream));
        ST_CUDA(c, cudaMemsetAsync(c->eLs.p, 0, P * 4, c->stream));
    }
    ST_CUDA(c, cudaStreamSynchronize(c->stream));   // the stacked values above are on the host
    c->np = P;
    c->ns = S;
    c->nb_total = NB;
    c->diffuse = false;
    c->pt.n = 0;          // the problems' particle trees stay in their parts
    c->et.n = 0;
    t.n = N;
    c->fr = c->bsub[0]->fr;
    c->fr.cmag = cmag;    // the filters' magnitude bound covers every problem
    c->nbatch = nb;
    c->built = true;
    return START_OK;
}

int start_set_state(start_ctx *c, const float *n_H, const double *y)
{
    if (!c) return START_EINVAL;
    if (!c->built) return set_err(c, START_ENOTBUILT, "start_build_trees first");
    DeviceGuard g(c);
    long long n = c->np;
    if (n && !n_H) return set_err(c, START_EINVAL, "NULL n_H");
    if (n == 0) {
        c->has_state = true;
        return START_OK;
    }
    unsigned long long *ctr = c->counters.as<unsigned long long>();
    Staged in;
    ST_TRY(stage_in(c, in.h, n_H, n * sizeof(float)));
    if (y) ST_TRY(stage_in(c, in.V, y, n * sizeof(double)));
    k_check_nonneg_f<<<grid_for(n, 256), 256, 0, c->stream>>>(in.h.as<float>(), n, ctr + C_BAD_INPUT); ++c->launches;
    if (y) { k_check_unit_d<<<grid_for(n, 256), 256, 0, c->stream>>>(in.V.as<double>(), n, ctr + C_BAD_INPUT); ++c->launches; }
    ST_TRY(check_bad(c, "n_H or y"));
    k_set_state<<<grid_for(n, 256), 256, 0, c->stream>>>(in.h.as<float>(), y ? in.V.as<double>() : nullptr,
                                                        c->pinv.as<u32>(), n, c->nH.as<float>(),
                                                        c->y.as<double>(), c->pq.as<float4>()); ++c->launches;
    k_fill_d<<<grid_for(n, 256), 256, 0, c->stream>>>(c->Tg.as<double>(), n, 1e4); ++c->launches;
    ST_CUDA(c, cudaGetLastError());
    ST_CUDA(c, cudaStreamSynchronize(c->stream));
    c->has_state = true;
    return START_OK;
}

int start_set_temperature(start_ctx *c, const double *T)
{
    if (!c) return START_EINVAL;
    if (!c->built) return set_err(c, START_ENOTBUILT, "start_build_trees first");
    DeviceGuard g(c);
    long long n = c->np;
    if (n == 0) return START_OK;
    if (!T) return set_err(c, START_EINVAL, "NULL T");
    unsigned long long *ctr = c->counters.as<unsigned long long>();
    Staged in;
    ST_TRY(stage_in(c, in.V, T, n * sizeof(double)));
    k_check_nonneg_d<<<grid_for(n, 256), 256, 0, c->stream>>>(in.V.as<double>(), n,
                                                              ctr + C_BAD_INPUT, 1);
    ++c->launches;
    ST_TRY(check_bad(c, "T"));
    k_scatter_d<<<grid_for(n, 256), 256, 0, c->stream>>>(in.V.as<double>(), c->pinv.as<u32>(), n,
                                                         c->Tg.as<double>());
    ++c->launches;
    ST_CUDA(c, cudaGetLastError());
    ST_CUDA(c, cudaStreamSynchronize(c->stream));
    return START_OK;
}

int start_get_temperature(start_ctx *c, double *T_out)
{
    if (!c || (!T_out && c->np > 0)) return START_EINVAL;
    if (!c->built) return set_err(c, START_ENOTBUILT, "start_build_trees first");
    DeviceGuard g(c);
    long long n = c->np;
    if (n == 0) return START_OK;
    ST_TRY(ensure(c->stage, n * sizeof(double)));
    k_to_input_order<double><<<grid_for(n, 256), 256, 0, c->stream>>>(
        c->Tg.as<double>(), c->porig.as<u32>(), n, c->stage.as<double>());
    ++c->launches;
    ST_CUDA(c, cudaGetLastError());
    return copy_out(c, T_out, c->stage.p, n * sizeof(double));
}

int start_rt_solve(start_ctx *c, const float *n_HI, float theta, float *gamma_out)
{
    if (!c) return START_EINVAL;
    if (!c->built) return set_err(c, START_ENOTBUILT, "start_build_trees first");
    if (!(theta >= 0.f) || !isfinite(theta)) return set_err(c, START_EINVAL, "theta must be >= 0");
    DeviceGuard g(c);
    long long n = c->np;
    if (n_HI && n) {
        Staged in;
        unsigned long long *ctr = c->counters.as<unsigned long long>();
        ST_TRY(stage_in(c, in.h, n_HI, n * sizeof(float)));
        k_check_nonneg_f<<<grid_for(n, 256), 256, 0, c->stream>>>(in.h.as<float>(), n, ctr + C_BAD_INPUT); ++c->launches;
        ST_TRY(check_bad(c, "n_HI"));
        k_set_nHI<<<grid_for(n, 256), 256, 0, c->stream>>>(in.h.as<float>(), c->pinv.as<u32>(), n,
                                                          c->pq.as<float4>()); ++c->launches;
        ST_CUDA(c, cudaGetLastError());
    } else if (!n_HI && c->diffuse && !c->has_state && n) {
        return set_err(c, START_ENOTBUILT, "diffuse mode needs start_set_state");
    }
    bool dev_out = gamma_out && is_device_ptr(gamma_out);
    if (gamma_out && !dev_out) ST_TRY(ensure(c->stage, (n ? n : 1) * sizeof(float)));
    float *gdst = dev_out ? gamma_out : (gamma_out ? c->stage.as<float>() : nullptr);
    if (c->p.reuse_chains && c->r_valid && c->r_theta == theta && !c->diffuse &&
        c->p.T_eff == 0.0) {
        c->heat_valid = false;
        phase_mark(c, START_PHASE_GAMMA, false);   // the whole step on resident chains
        ST_TRY(resident_solve(c));
        if (gdst && n) {
            k_to_input_order<float><<<grid_for(n, 256), 256, 0, c->stream>>>(
                c->gam.as<float>(), c->porig.as<u32>(), n, gdst);
            ++c->launches;
            ST_CUDA(c, cudaGetLastError());
        }
        phase_mark(c, START_PHASE_GAMMA, true);
    } else {
        ST_TRY(run_solve(c, theta, gdst));
        if (resident_eligible(c)) ST_TRY(resident_build(c, theta));
    }
    if (gamma_out && !dev_out) ST_TRY(copy_out(c, gamma_out, c->stage.p, n * sizeof(float)));
    ST_CUDA(c, cudaStreamSynchronize(c->stream));
    if (read_counter(c, C_INTERNAL)) return set_err(c, START_ECUDA, "internal inconsistency (interaction lists)");
    if (read_counter(c, C_CHAIN_OVF)) return set_err(c, START_ECHAIN, "a ray exceeded hop_cap");
    c->solved = true;
    return START_OK;
}

int start_ionize(start_ctx *c, double dt_s, double *y_out)
{
    if (!c) return START_EINVAL;
    if (!c->built || !c->solved) return set_err(c, START_ENOTBUILT, "start_rt_solve first");
    if (!(dt_s >= 0.0) || !isfinite(dt_s)) return set_err(c, START_EINVAL, "dt must be >= 0");
    DeviceGuard g(c);
    if (c->p.thermal) ST_TRY(run_ionize_thermal(c, dt_s));
    else ST_TRY(run_ionize(c, dt_s));
    if (y_out && c->np) {
        bool dev = is_device_ptr(y_out);
        double *dst = y_out;
        if (!dev) {
            ST_TRY(ensure(c->stage, c->np * sizeof(double)));
            dst = c->stage.as<double>();
        }
        k_to_input_order<double><<<grid_for(c->np, 256), 256, 0, c->stream>>>(
            c->y.as<double>(), c->porig.as<u32>(), c->np, dst); ++c->launches;
        ST_CUDA(c, cudaGetLastError());
        if (!dev) ST_TRY(copy_out(c, y_out, dst, c->np * sizeof(double)));
    }
    return START_OK;
}

int start_sph_density(start_ctx *c, const float *mass, float *rho_out)
{
    if (!c) return START_EINVAL;
    if (!c->built) return set_err(c, START_ENOTBUILT, "start_build_trees first");
    long long n = c->np;
    if (n && (!mass || !rho_out)) return set_err(c, START_EINVAL, "NULL mass or rho_out");
    if (n == 0) return START_OK;
    DeviceGuard g(c);
    const float *md = mass;
    if (!is_device_ptr(mass)) {
        ST_TRY(stage_in(c, c->mass_in, mass, n * sizeof(float)));
        md = c->mass_in.as<float>();
    }
    bool dev_out = is_device_ptr(rho_out);
    float *dst = rho_out;
    if (!dev_out) {
        ST_TRY(ensure(c->stage, n * sizeof(float)));
        dst = c->stage.as<float>();
    }
    ST_TRY(run_sph_density(c, md, dst));
    ST_TRY(check_bad(c, "mass (must be finite and >= 0)"));
    if (!dev_out) ST_TRY(copy_out(c, rho_out, dst, n * sizeof(float)));
    return START_OK;
}

int start_get_heating(start_ctx *c, float *heat_out)
{
    if (!c) return START_EINVAL;
    if (!c->solved) return set_err(c, START_ENOTBUILT, "start_rt_solve first");
    long long n = c->np;
    if (n && !heat_out) return set_err(c, START_EINVAL, "NULL heat_out");
    if (n == 0) return START_OK;
    DeviceGuard g(c);
    bool dev = is_device_ptr(heat_out);
    float *dst = heat_out;
    if (!dev) {
        ST_TRY(ensure(c->stage, n * sizeof(float)));
        dst = c->stage.as<float>();
    }
    if (c->heat_valid) {
        k_to_input_order<float><<<grid_for(n, 256), 256, 0, c->stream>>>(
            c->heat.as<float>(), c->porig.as<u32>(), n, dst);
        ++c->launches;
        ST_CUDA(c, cudaGetLastError());
    } else {
        ST_CUDA(c, cudaMemsetAsync(dst, 0, n * sizeof(float), c->stream));
    }
    if (!dev) ST_TRY(copy_out(c, heat_out, dst, n * sizeof(float)));
    return START_OK;
}

int start_h2_dissociation(start_ctx *c, const float *n_H2, float theta, double kappa_LW,
                          float *kdis_out)
{
    if (!c) return START_EINVAL;
    if (!c->built) return set_err(c, START_ENOTBUILT, "start_build_trees first");
    if (!(theta >= 0.f) || !isfinite(theta)) return set_err(c, START_EINVAL, "theta must be >= 0");
    if (!(kappa_LW >= 0.0) || !isfinite(kappa_LW))
        return set_err(c, START_EINVAL, "kappa_LW must be finite and >= 0");
    long long n = c->np;
    if (n && (!n_H2 || !kdis_out)) return set_err(c, START_EINVAL, "NULL n_H2 or kdis_out");
    if (n == 0) return START_OK;
    DeviceGuard g(c);
    const float *nd = n_H2;
    if (!is_device_ptr(n_H2)) {
        ST_TRY(stage_in(c, c->h2_in, n_H2, n * sizeof(float)));
        nd = c->h2_in.as<float>();
    }
    bool dev_out = is_device_ptr(kdis_out);
    float *dst = kdis_out;
    if (!dev_out) {
        ST_TRY(ensure(c->stage, n * sizeof(float)));
        dst = c->stage.as<float>();
    }
    c->kappa_LW = kappa_LW;
    ST_TRY(run_h2_dissociation(c, nd, theta, dst));
    ST_CUDA(c, cudaStreamSynchronize(c->stream));
    if (read_counter(c, C_INTERNAL)) return set_err(c, START_ECUDA, "internal inconsistency");
    if (read_counter(c, C_CHAIN_OVF)) return set_err(c, START_ECHAIN, "a ray exceeded hop_cap");
    if (!dev_out) ST_TRY(copy_out(c, kdis_out, dst, n * sizeof(float)));
    return START_OK;
}

int start_rt_solve_oneshot(const start_params *p, const float *pos, const float *h, long long n_p,
                           const float *n_HI, const float *src_pos, const double *src_L,
                           long long n_s, float theta, float *gamma_out)
{
    start_ctx *c = nullptr;
    int rc = start_create(&c, p);
    if (rc) return rc;
    rc = start_build_trees(c, pos, h, n_p, src_pos, src_L, n_s, nullptr, 0);
    if (!rc && n_p) rc = n_HI ? START_OK : START_EINVAL;
    if (!rc) rc = start_rt_solve(c, n_HI, theta, gamma_out);
    if (!rc) cudaStreamSynchronize(c->stream);
    start_destroy(c);
    return rc;
}

int start_get_frame(start_ctx *c, double out[4])
{
    if (!c || !out) return START_EINVAL;
    if (!c->built) return set_err(c, START_ENOTBUILT, "start_build_trees first");
    for (int a = 0; a < 3; ++a) out[a] = c->fr.lo[a];
    out[3] = c->fr.side;
    return START_OK;
}

int start_get_perm(start_ctx *c, int which, unsigned *perm)
{
    if (!c || !perm || (which != 0 && which != 1)) return START_EINVAL;
    if (!c->built) return set_err(c, START_ENOTBUILT, "start_build_trees first");
    DeviceGuard g(c);
    long long n = which ? c->ns : c->np;
    return copy_out(c, perm, which ? c->sorig.p : c->porig.p, n * sizeof(u32));
}

int start_get_keys(start_ctx *c, int which, unsigned long long *keys)
{
    if (!c || !keys || (which != 0 && which != 1)) return START_EINVAL;
    if (!c->built) return set_err(c, START_ENOTBUILT, "start_build_trees first");
    DeviceGuard g(c);
    long long n = which ? c->ns : c->np;
    return copy_out(c, keys, which ? c->skey.p : c->pkey.p, n * sizeof(u64));
}

static Tree *pick_tree(start_ctx *c, int which)
{
    return which == 0 ? &c->pt : which == 1 ? &c->stree : which == 2 ? &c->et : nullptr;
}

long long start_tree_size(start_ctx *c, int which)
{
    if (!c || !pick_tree(c, which)) return START_EINVAL;
    if (!c->built) return set_err(c, START_ENOTBUILT, "start_build_trees first");
    return pick_tree(c, which)->n;
}

int start_get_tree(start_ctx *c, int which, int *level, unsigned *first, unsigned *count,
                   unsigned *skip, int *leaf, double *cube4, double *L, float *cen3)
{
    Tree *t = c ? pick_tree(c, which) : nullptr;
    if (!t) return START_EINVAL;
    if (!c->built) return set_err(c, START_ENOTBUILT, "start_build_trees first");
    DeviceGuard g(c);
    long long n = t->n;
    if (n == 0) return START_OK;
    if (which == 2 && c->diffuse && c->has_state) ST_TRY(refresh_emitters(c));
    std::vector<uint4> meta(n);
    ST_CUDA(c, cudaMemcpyAsync(meta.data(), t->meta.p, n * sizeof(uint4), cudaMemcpyDeviceToHost,
                               c->stream));
    ST_CUDA(c, cudaStreamSynchronize(c->stream));
    std::vector<unsigned> a(n), b(n), d(n);
    std::vector<int> lf(n);
    for (long long i = 0; i < n; ++i) {
        d[i] = meta[i].x;
        a[i] = meta[i].y;
        b[i] = meta[i].z;
        lf[i] = (int)meta[i].w;
    }
    ST_TRY(copy_out(c, level, t->level.p, n * sizeof(int)));
    ST_CUDA(c, cudaStreamSynchronize(c->stream));
    if (first) ST_CUDA(c, cudaMemcpy(first, a.data(), n * 4, cudaMemcpyDefault));
    if (count) ST_CUDA(c, cudaMemcpy(count, b.data(), n * 4, cudaMemcpyDefault));
    if (skip) ST_CUDA(c, cudaMemcpy(skip, d.data(), n * 4, cudaMemcpyDefault));
    if (leaf) ST_CUDA(c, cudaMemcpy(leaf, lf.data(), n * 4, cudaMemcpyDefault));
    ST_TRY(copy_out(c, cube4, t->cube.p, n * 4 * sizeof(double)));
    bool has_mom = which != 0 && t->L.p && t->vsrc.p;
    if (L) {
        if (has_mom) ST_TRY(copy_out(c, L, t->L.p, n * sizeof(double)));
        else ST_CUDA(c, cudaMemset(L, 0, n * sizeof(double)));
    }
    if (cen3) {
        std::vector<float4> v(n);
        if (has_mom) {
            ST_CUDA(c, cudaMemcpyAsync(v.data(), t->vsrc.p, n * sizeof(float4),
                                       cudaMemcpyDeviceToHost, c->stream));
            ST_CUDA(c, cudaStreamSynchronize(c->stream));
        } else {
            memset(v.data(), 0, n * sizeof(float4));
        }
        std::vector<float> cc(3 * n);
        for (long long i = 0; i < n; ++i) {
            cc[3 * i] = v[i].x;
            cc[3 * i + 1] = v[i].y;
            cc[3 * i + 2] = v[i].z;
        }
        ST_CUDA(c, cudaMemcpy(cen3, cc.data(), 3 * n * sizeof(float), cudaMemcpyDefault));
    }
    return START_OK;
}

long long start_nbr_total(start_ctx *c)
{
    if (!c) return START_EINVAL;
    if (!c->built) return set_err(c, START_ENOTBUILT, "start_build_trees first");
    return c->nb_total;
}

int start_get_neighbors(start_ctx *c, unsigned long long *off, unsigned *idx)
{
    if (!c || !off) return START_EINVAL;
    if (!c->built) return set_err(c, START_ENOTBUILT, "start_build_trees first");
    DeviceGuard g(c);
    long long n = c->np;
    ST_CUDA(c, cudaStreamSynchronize(c->stream));
    std::vector<u32> moff(n + 1), mval(c->nb_total), porig(n);
    ST_CUDA(c, cudaMemcpy(moff.data(), c->nb_off.p, (n + 1) * 4, cudaMemcpyDeviceToHost));
    if (c->nb_total) ST_CUDA(c, cudaMemcpy(mval.data(), c->nb_idx.p, c->nb_total * 4, cudaMemcpyDeviceToHost));
    if (n) ST_CUDA(c, cudaMemcpy(porig.data(), c->porig.p, n * 4, cudaMemcpyDeviceToHost));
    std::vector<u64> o;
    std::vector<u32> v;
    csr_to_input<u32>(n, moff, mval, porig, true, o, v);
    ST_CUDA(c, cudaMemcpy(off, o.data(), (n + 1) * 8, cudaMemcpyDefault));
    if (idx && !v.empty()) ST_CUDA(c, cudaMemcpy(idx, v.data(), v.size() * 4, cudaMemcpyDefault));
    return START_OK;
}

int start_get_lists(start_ctx *c, float theta, unsigned long long *off, unsigned *entries)
{
    if (!c || !off) return START_EINVAL;
    if (!c->built) return set_err(c, START_ENOTBUILT, "start_build_trees first");
    if (!(theta >= 0.f) || !isfinite(theta)) return set_err(c, START_EINVAL, "theta must be >= 0");
    DeviceGuard g(c);
    long long n = c->np;
    if (c->diffuse && c->has_state) ST_TRY(refresh_emitters(c));
    ST_TRY(run_walk(c, theta));
    ST_CUDA(c, cudaStreamSynchronize(c->stream));
    std::vector<u64> moff(n + 1);
    std::vector<u32> mval(c->npairs), porig(n);
    ST_CUDA(c, cudaMemcpy(moff.data(), c->loff.p, (n + 1) * 8, cudaMemcpyDeviceToHost));
    if (c->npairs) ST_CUDA(c, cudaMemcpy(mval.data(), c->pent.p, c->npairs * 4, cudaMemcpyDeviceToHost));
    if (n) ST_CUDA(c, cudaMemcpy(porig.data(), c->porig.p, n * 4, cudaMemcpyDeviceToHost));
    std::vector<u64> o;
    std::vector<u32> v;
    csr_to_input<u64>(n, moff, mval, porig, false, o, v);
    ST_CUDA(c, cudaMemcpy(off, o.data(), (n + 1) * 8, cudaMemcpyDefault));
    if (entries && !v.empty()) ST_CUDA(c, cudaMemcpy(entries, v.data(), v.size() * 4, cudaMemcpyDefault));
    return START_OK;
}

int start_get_list_hashes(start_ctx *c, float theta, unsigned long long *hash,
                          unsigned long long *count)
{
    if (!c || (!hash && c->np > 0)) return START_EINVAL;
    if (!c->built) return set_err(c, START_ENOTBUILT, "start_build_trees first");
    if (!(theta >= 0.f) || !isfinite(theta)) return set_err(c, START_EINVAL, "theta must be >= 0");
    DeviceGuard g(c);
    long long n = c->np;
    if (n == 0) return START_OK;
    if (c->diffuse && c->has_state) ST_TRY(refresh_emitters(c));
    ST_TRY(ensure(c->stage, (size_t)n * 16));
    unsigned long long *dh = c->stage.as<unsigned long long>();
    ST_TRY(run_walk_hash(c, theta, dh, dh + n));
    ST_TRY(copy_out(c, hash, dh, (size_t)n * 8));
    if (count) ST_TRY(copy_out(c, count, dh + n, (size_t)n * 8));
    return START_OK;
}

int start_get_emitter_L(start_ctx *c, float *out)
{
    if (!c || !out) return START_EINVAL;
    if (!c->built) return set_err(c, START_ENOTBUILT, "start_build_trees first");
    DeviceGuard g(c);
    if (c->np == 0) return START_OK;
    if (c->diffuse && c->has_state) ST_TRY(refresh_emitters(c));
    ST_TRY(ensure(c->stage, c->np * sizeof(float)));
    k_to_input_order<float><<<grid_for(c->np, 256), 256, 0, c->stream>>>(
        c->eLs.as<float>(), c->porig.as<u32>(), c->np, c->stage.as<float>()); ++c->launches;
    ST_CUDA(c, cudaGetLastError());
    return copy_out(c, out, c->stage.p, c->np * sizeof(float));
}

int start_get_stats(start_ctx *c, start_stats *out)
{
    if (!c || !out) return START_EINVAL;
    DeviceGuard g(c);
    unsigned long long v[C_COUNT];
    ST_CUDA(c, cudaMemcpyAsync(v, c->counters.p, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
    ST_CUDA(c, cudaStreamSynchronize(c->stream));
    memset(out, 0, sizeof(*out));
    // the memoised march counts chain links only in the counting form
    const bool counted = c->hops_counted;
    out->rays = (long long)v[C_RAYS];
    out->hops = counted ? (long long)v[C_HOPS] : -1;
    out->march_fallbacks = (long long)v[C_MARCH_FB];
    out->walk_fallbacks = (long long)v[C_WALK_FB];
    out->nbr_fallbacks = (long long)v[C_NBR_FB];
    out->max_hops = counted ? (long long)v[C_MAX_HOPS] : -1;
    out->nodes_src = c->stree.n;
    out->nodes_emit = c->et.n;
    out->nodes_part = c->pt.n;
    out->nbr_total = c->nb_total;
    out->launches = (long long)c->launches;
    out->evals = (long long)v[C_EVALS];
    out->links = (long long)(c->p.march_mode == 1 ? v[C_SLOTS] : 0);
    out->chunks = c->chunks;
    out->jump_rounds = c->jump_rounds;
    out->jump_bytes = (long long)c->jump_bytes;
    out->first_hop_scanned = (long long)v[C_ROW_CAND];
    out->first_hop_full = (long long)v[C_ROW_NB];
    return START_OK;
}

int start_get_timings(start_ctx *c, double *ms, int n)
{
    if (!c || !ms || n < 0 || n > START_NPHASES) return START_EINVAL;
    DeviceGuard g(c);
    ST_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < n; ++k) {
        ms[k] = -1.0;
        if (k == START_PHASE_HOPS || k == START_PHASE_LINK || k == START_PHASE_JUMP) {
            double v = k == START_PHASE_HOPS ? c->hop_ms
                       : k == START_PHASE_LINK ? c->link_ms : c->jump_ms;
            if (c->p.timing && c->p.march_mode == 1) ms[k] = v;
            continue;
        }
        if (c->pcount[k] == 0) continue;
        double sum = 0.0;
        for (int q = 0; q < c->pcount[k]; ++q) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, c->pev[k][2 * q], c->pev[k][2 * q + 1]) == cudaSuccess)
                sum += t;
            else
                cudaGetLastError();
        }
        ms[k] = sum;
    }
    for (int k = 0; k < START_NPHASES; ++k) c->pcount[k] = 0;
    c->hop_ms = c->link_ms = c->jump_ms = 0.0;
    return START_OK;
}

const char *start_last_error(const start_ctx *c)
{
    if (!c) return "NULL context";
    return c->err.c_str();
}

long long start_memory_in_use(void) { return bytes_in_use(); }

int start_direction_bins(int N, float *cones)
{
    if (N < 2 || N > 6 || !cones) return START_EINVAL;
    direction_bin_cones(N, cones);
    return START_OK;
}

const char *start_status_string(int s)
{
    switch (s) {
    case START_OK: return "START_OK";
    case START_EINVAL: return "START_EINVAL";
    case START_ENOMEM: return "START_ENOMEM";
    case START_ENOTBUILT: return "START_ENOTBUILT";
    case START_ECUDA: return "START_ECUDA";
    case START_ETIMEOUT: return "START_ETIMEOUT";
    case START_ECHAIN: return "START_ECHAIN";
    case START_ERANGE: return "START_ERANGE";
    default: return "START_E?";
    }
}

}  // extern "C"
