// C-ABI layer of libens: context, device memory layout, stream/graph
// orchestration of the hot-path kernels, host<->device marshalling.
#include "../../include/ens.h"
#include "ens_launch.h"
#include "ens_persist.h"

#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace ens;

namespace {

constexpr size_t kAlign = 256;

struct Group {
    Geo geo;
    std::vector<int> members;   // global member indices, in order
};

struct Arena {
    char *base;
    size_t off = 0;
    template <class T>
    T *take(size_t count)
    {
        off = (off + kAlign - 1) / kAlign * kAlign;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += sizeof(T) * count;
        return p;
    }
};

int kc_of(int N) { return (N + 2) / 3 - 1; }

}  // namespace

struct ens_ctx {
    std::vector<ens_member_desc> desc;
    ens_hist_spec hist{};
    std::vector<Group> groups;
    std::vector<int> member_group, member_local;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    std::vector<cudaStream_t> aux;        // one per group (index 0 unused)
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
    void *workspace = nullptr;
    bool owns = false;
    size_t ws_bytes = 0;
    MemberDev *md = nullptr;
    double *partial = nullptr;
    int partial_blocks = 0;
    unsigned long long *counts = nullptr;
    double *moments = nullptr;
    double *mom_partial = nullptr;
    int mom_blocks = 0;
    float *edges = nullptr;
    HistDev hd{};
    double *mix = nullptr;       // mixture scratch
    cudaGraphExec_t graph = nullptr;
    // streamed host step: copy streams and per-chunk events (created on first use)
    cudaStream_t copy_in = nullptr, copy_out = nullptr;
    cudaEvent_t ev_start = nullptr;
    std::vector<cudaEvent_t> ev_in, ev_done;
    int rk = 3;
    int sms = 0;                 // streaming multiprocessors of the device
    int parallel_groups = 1;     // grid-size groups as parallel graph branches
    int skip_member = -1;        // ens_test_skip_copy: member armed for the next ens_step_nograph (-1: none)
    // persistent stage kernel (grid sizes 128, 256, 384): work items, counters
    PItem *pitems = nullptr;
    int npitems = 0;
    unsigned *pwork = nullptr;   // [2 + members * kPKinds]: item counter, abort flag, per-member done counts
    unsigned pneed[kPSlots][kPKinds] = {};
    int persist_ctas = 0;        // resident CTAs of the persistent kernel (0: unavailable)
    int persistent = 0;          // 1: one persistent launch per RK stage
    int skip_wait = 0;
    ens_status sticky = ENS_OK;
    std::string err;
};

namespace {

ens_status fail(ens_ctx *ctx, ens_status s, const std::string &msg)
{
    if (ctx && ctx->sticky == ENS_OK) {
        ctx->sticky = s;
        ctx->err = msg;
    }
    return s;
}

ens_status cuda_fail(ens_ctx *ctx, const char *what, cudaError_t e)
{
    return fail(ctx, ENS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define ENS_CUDA(ctx, call)                                   \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) return cuda_fail(ctx, #call, _e); \
    } while (0)

ens_status validate_hist(const ens_hist_spec *h, std::string &why)
{
    if (h->qr_bins < 1 || h->qr_bins > 256 || h->tail_bins < 1 || h->tail_bins > 4096) { why = "histogram bins out of range"; return ENS_EINVAL; }
    if (h->grad_bins < 0 || h->grad_bins > 2048 || (h->grad_bins > 0 && !(h->grad_lim > 0 && std::isfinite(h->grad_lim)))) {
        why = "gradient-component histogram: 0 <= grad_bins <= 2048 and grad_lim > 0";
        return ENS_EINVAL;
    }
    if (!(h->q_lim > 0) || !(h->r_lim > 0) || !(h->tail_hi > h->tail_lo) || !(h->eps_norm > 0) || !(h->nu_norm > 0)) {
        why = "invalid histogram ranges or normalisation";
        return ENS_EINVAL;
    }
    return ENS_OK;
}

ens_status validate(const ens_member_desc *m, int n, const ens_hist_spec *h, std::string &why)
{
    if (!m || n <= 0) { why = "no members"; return ENS_EINVAL; }
    if (n > 1024) { why = "at most 1024 members"; return ENS_EINVAL; }
    if (!h) { why = "no histogram specification"; return ENS_EINVAL; }
    for (int i = 0; i < n; ++i) {
        const ens_member_desc &d = m[i];
        char buf[160];
        if (!supported_n(d.N)) {
            snprintf(buf, sizeof buf, "member %d: N=%d has no FFT plan (16,32,64,128,256,384,512)", i, d.N);
            why = buf;
            return ENS_EUNSUPPORTED;
        }
        const int kc = kc_of(d.N);
        if (d.rk_order != 2 && d.rk_order != 3) { snprintf(buf, sizeof buf, "member %d: rk_order must be 2 or 3", i); why = buf; return ENS_EINVAL; }
        if (d.rk_order != m[0].rk_order) { why = "all members must share rk_order"; return ENS_EINVAL; }
        if (!(d.nu > 0.0) || !(d.eps_bar > 0.0) || !std::isfinite(d.lambda)) { snprintf(buf, sizeof buf, "member %d: nu, eps_bar must be > 0 and lambda finite", i); why = buf; return ENS_EINVAL; }
        if (!(d.k_lo >= 0.0) || !(d.k_hi >= d.k_lo) || d.k_hi > kc + 1e-9) {
            snprintf(buf, sizeof buf, "member %d: band [%g, %g] must lie inside the dealiased set |k| <= %d", i, d.k_lo, d.k_hi, kc);
            why = buf;
            return ENS_EINVAL;
        }
        {
            // the band must hold a wave vector other than k = 0: an integer
            // k^2 >= 1 in [k_lo^2, k_hi^2] that is a sum of three squares (not
            // of the form 4^a (8 b + 7)); its components are <= |k| <= kc, so
            // the mode is kept.  Otherwise E_B = 0 and the forcing is undefined.
            const long long lo2 = std::max(1LL, (long long)std::ceil(d.k_lo * d.k_lo - 1e-9));
            const long long hi2 = (long long)std::floor(d.k_hi * d.k_hi + 1e-9);
            bool any = false;
            for (long long q = lo2; q <= hi2 && !any; ++q) {
                long long r = q;
                while (r % 4 == 0) r /= 4;
                any = r % 8 != 7;
            }
            if (!any) {
                snprintf(buf, sizeof buf, "member %d: band [%g, %g] holds no wave vector besides k = 0", i, d.k_lo, d.k_hi);
                why = buf;
                return ENS_EINVAL;
            }
        }
        if (!(d.dt > 0.0) && !(d.cfl > 0.0)) { snprintf(buf, sizeof buf, "member %d: need dt > 0 or cfl > 0", i); why = buf; return ENS_EINVAL; }
        if (!(d.init_energy > 0.0)) { snprintf(buf, sizeof buf, "member %d: init_energy must be > 0", i); why = buf; return ENS_EINVAL; }
    }
    return validate_hist(h, why);
}

// Group members by N (ascending), carve the workspace (base == nullptr: size only).
size_t carve(const ens_member_desc *m, int n, const ens_hist_spec *h, char *base, ens_ctx *ctx)
{
    Arena ar{base};
    std::vector<int> Ns;
    for (int i = 0; i < n; ++i) Ns.push_back(m[i].N);
    std::sort(Ns.begin(), Ns.end());
    Ns.erase(std::unique(Ns.begin(), Ns.end()), Ns.end());
    MemberDev *md = ar.take<MemberDev>(n);
    std::vector<Group> groups;
    int PB = 1, MB = 1;
    int first = 0;
    for (int N : Ns) {
        Group gr;
        for (int i = 0; i < n; ++i)
            if (m[i].N == N) gr.members.push_back(i);
        Geo &g = gr.geo;
        g.N = N;
        g.kc = kc_of(N);
        g.NK = 2 * g.kc + 1;
        g.NZ = g.kc + 1;
        g.NZp = (g.NZ + kTile - 1) / kTile * kTile;
        g.tile_x = g.tile_y = kTile;
        g.plan_x = 0;
        g.fx_split = 0;
        g.z_mode = 0;
        g.z_skip_member = -1;
        g.z_skip_wait = 0;
        g.members = (int)gr.members.size();
        g.first = first;
        first += g.members;
        g.sU = (long long)g.NK * g.NK * g.NZp;
        g.sA = (long long)g.NK * N * g.NZp;
        g.sB = (long long)N * N * g.NZp;
        g.tw = ar.take<float2>(N);
        g.U = ar.take<float2>(3 * g.sU * g.members);
        g.S = ar.take<float2>(3 * g.sU * g.members);
        g.A = ar.take<float2>((size_t)kFields * g.sA * g.members);
        g.B = ar.take<float2>((size_t)kFields * g.sB * g.members);
        g.shells = (int)std::ceil(std::sqrt(3.0) * g.kc) + 2;
        g.shell = ar.take<double>((size_t)g.shells * g.members);
        PB = std::max(PB, g.NK * g.NZp / 8);   // narrowest column tile of the update pass
        PB = std::max(PB, (int)((g.sU + kUpdChunk - 1) / kUpdChunk));   // split update pass
        MB = std::max(MB, stats_blocks(N));
        groups.push_back(gr);
    }
    const long long L = counts_len_of(h->qr_bins, h->tail_bins, h->grad_bins);
    double *partial = ar.take<double>((size_t)n * PB * 4);
    unsigned long long *counts = ar.take<unsigned long long>((size_t)n * L);
    double *moments = ar.take<double>((size_t)n * kNMom);
    double *mom_partial = ar.take<double>((size_t)n * MB * kNMom);
    float *edges = ar.take<float>((size_t)2 * (h->qr_bins + 1) + h->tail_bins + 1 + h->grad_bins + 1);
    // mixture scratch: lambdas, user weights, weights, covered, pdf, mixed moments, ratios
    double *mix = ar.take<double>((size_t)3 * n + 1 + L + kNMom + 8);
    // work items of the persistent stage kernel, where every grid size has its pass bodies there
    PItem *pitems = nullptr;
    unsigned *pwork = nullptr;
    int npitems = 0;
    unsigned pneed[kPSlots][kPKinds];
    bool persist = groups.size() <= (size_t)kPSlots;
    for (auto &gr : groups) persist = persist && persist_size_supported(gr.geo.N);
    if (persist) {
        std::vector<Geo> geos;
        for (auto &gr : groups) geos.push_back(gr.geo);
        std::vector<PItem> items;
        persist_items(geos, items, pneed);
        npitems = (int)items.size();
        pitems = ar.take<PItem>(items.size());
        pwork = ar.take<unsigned>(2 + (size_t)n * kPKinds);
    }
    if (ctx) {
        ctx->pitems = persist ? pitems : nullptr;
        ctx->npitems = npitems;
        ctx->pwork = pwork;
        if (persist) std::memcpy(ctx->pneed, pneed, sizeof pneed);
        ctx->md = md;
        ctx->partial = partial;
        ctx->partial_blocks = PB;
        ctx->counts = counts;
        ctx->moments = moments;
        ctx->mom_partial = mom_partial;
        ctx->mom_blocks = MB;
        ctx->edges = edges;
        ctx->mix = mix;
        ctx->member_group.assign(n, 0);
        ctx->member_local.assign(n, 0);
        // renumber: members are stored group by group (global index = g.first + local)
        for (size_t gi = 0; gi < groups.size(); ++gi) {
            Geo &g = groups[gi].geo;
            g.partial = partial;
            g.partial_blocks = PB;
            g.counts = counts;
            g.mom_partial = mom_partial;
            g.mom_blocks = MB;
            for (int k = 0; k < g.members; ++k) {
                ctx->member_group[groups[gi].members[k]] = (int)gi;
                ctx->member_local[groups[gi].members[k]] = k;
            }
        }
        ctx->groups = groups;
    }
    return ar.off + kAlign;
}

// device slot of user member i
int slot_of(const ens_ctx *ctx, int i) { return ctx->groups[ctx->member_group[i]].geo.first + ctx->member_local[i]; }

// Members [k0, k0 + cnt) of a group (pointers shifted).
Geo member_range(const Geo &g0, int k0, int cnt)
{
    Geo g = g0;
    g.U += (long long)k0 * 3 * g.sU;
    g.S += (long long)k0 * 3 * g.sU;
    g.A += (long long)k0 * kFields * g.sA;
    g.B += (long long)k0 * kFields * g.sB;
    g.shell += (long long)k0 * g.shells;
    g.first += k0;
    g.members = cnt;
    return g;
}

// Geo restricted to one member of a group (pointers shifted).
Geo single(const ens_ctx *ctx, int i)
{
    Geo g = ctx->groups[ctx->member_group[i]].geo;
    const int k = ctx->member_local[i];
    g.U += (long long)k * 3 * g.sU;
    g.S += (long long)k * 3 * g.sU;
    g.A += (long long)k * kFields * g.sA;
    g.B += (long long)k * kFields * g.sB;
    g.shell += (long long)k * g.shells;
    g.first += k;
    g.members = 1;
    return g;
}

void record_group_stage(ens_ctx *ctx, const Geo &g, int st, int last, cudaStream_t s)
{
    launch_pass(Pass::IX, 0, g, ctx->md, nullptr, st, last, st > 0 ? 1 : 0, s);
    launch_pass(Pass::IY, 0, g, ctx->md, nullptr, st, last, 6, s);
    launch_pass(Pass::Z, 0, g, ctx->md, nullptr, st, last, 0, s);
    launch_pass(Pass::FY, 0, g, ctx->md, nullptr, st, last, 0, s);
    launch_pass(Pass::FX, 0, g, ctx->md, nullptr, st, last, 0, s);
}

// One step with the persistent stage kernel: per RK stage, the work counters
// cleared and one cooperative launch that runs every pass of every member.
void record_step_persistent(ens_ctx *ctx, cudaStream_t s)
{
    const int n = (int)ctx->desc.size();
    PStageArgs a{};
    for (size_t gi = 0; gi < ctx->groups.size(); ++gi) a.g[gi] = ctx->groups[gi].geo;
    a.md = ctx->md;
    a.items = ctx->pitems;
    a.nitems = ctx->npitems;
    a.next = ctx->pwork;
    a.abort = ctx->pwork + 1;
    a.done = ctx->pwork + 2;
    std::memcpy(a.need, ctx->pneed, sizeof a.need);
    for (int st = 0; st < ctx->rk; ++st) {
        a.stage = st;
        a.last = st == ctx->rk - 1;
        cudaMemsetAsync(ctx->pwork, 0, sizeof(unsigned) * (2 + (size_t)n * kPKinds), s);
        launch_stage_persist(a, ctx->persist_ctas, s);
    }
}

// One step.  Groups of different grid size are independent until the
// per-member stage reduction, so with several groups each group's pass chain
// runs on its own stream (a parallel branch of the captured graph), joined
// before the reduction of every stage.
void record_step(ens_ctx *ctx, cudaStream_t s)
{
    if (ctx->persistent) {
        record_step_persistent(ctx, s);
        return;
    }
    const int nst = ctx->rk;
    const int n = (int)ctx->desc.size();
    const int ng = (int)ctx->groups.size();
    for (int st = 0; st < nst; ++st) {
        const int last = st == nst - 1;
        if (ng == 1 || !ctx->parallel_groups) {
            for (int gi = 0; gi < ng; ++gi) record_group_stage(ctx, ctx->groups[gi].geo, st, last, s);
        } else {
            cudaEventRecord(ctx->ev_fork, s);
            for (int gi = 1; gi < ng; ++gi) {
                cudaStreamWaitEvent(ctx->aux[gi], ctx->ev_fork, 0);
                record_group_stage(ctx, ctx->groups[gi].geo, st, last, ctx->aux[gi]);
                cudaEventRecord(ctx->ev_join[gi], ctx->aux[gi]);
            }
            record_group_stage(ctx, ctx->groups[0].geo, st, last, s);
            for (int gi = 1; gi < ng; ++gi) cudaStreamWaitEvent(s, ctx->ev_join[gi], 0);
        }
        launch_finish(ctx->md, n, ctx->partial, ctx->partial_blocks, st, last, 0, s);
    }
}

// Comparison mode: every member on its own, one after another, one stream.
void record_step_sequential(ens_ctx *ctx, cudaStream_t s)
{
    const int nst = ctx->rk;
    const int n = (int)ctx->desc.size();
    for (int st = 0; st < nst; ++st) {
        const int last = st == nst - 1;
        for (int i = 0; i < n; ++i) record_group_stage(ctx, single(ctx, i), st, last, s);
        launch_finish(ctx->md, n, ctx->partial, ctx->partial_blocks, st, last, 0, s);
    }
}

ens_status resum(ens_ctx *ctx)
{
    // partial slots the sums kernel does not write must read as zero
    ENS_CUDA(ctx, cudaMemsetAsync(ctx->partial, 0, sizeof(double) * ctx->desc.size() * ctx->partial_blocks * 4,
                                  ctx->stream));
    for (auto &gr : ctx->groups) launch_state_sums(gr.geo, ctx->md, ctx->stream);
    launch_finish(ctx->md, (int)ctx->desc.size(), ctx->partial, ctx->partial_blocks, 0, 0, 1, ctx->stream);
    ENS_CUDA(ctx, cudaGetLastError());
    return ENS_OK;
}

ens_status check(ens_ctx *ctx)
{
    if (!ctx) return ENS_EINVAL;
    return ctx->sticky;
}

void to_full(const ens_ctx *ctx, int i, const float2 *compact, double *full)
{
    const Geo &g = ctx->groups[ctx->member_group[i]].geo;
    const int N = g.N, H = N / 2 + 1;
    const size_t L = (size_t)N * N * H;
    std::memset(full, 0, sizeof(double) * 2 * 3 * L);
    for (int q = 0; q < 3; ++q)
        for (int ix = 0; ix < g.NK; ++ix)
            for (int iy = 0; iy < g.NK; ++iy)
                for (int kz = 0; kz < g.NZ; ++kz) {
                    const int kx = ix <= g.kc ? ix : ix - g.NK, ky = iy <= g.kc ? iy : iy - g.NK;
                    const size_t dst = q * L + ((size_t)((kx + N) % N) * N + (ky + N) % N) * H + kz;
                    const float2 v = compact[q * g.sU + ((size_t)ix * g.NK + iy) * g.NZp + kz];
                    full[2 * dst] = v.x;
                    full[2 * dst + 1] = v.y;
                }
}

void from_full(const ens_ctx *ctx, int i, const double *full, float2 *compact)
{
    const Geo &g = ctx->groups[ctx->member_group[i]].geo;
    const int N = g.N, H = N / 2 + 1;
    const size_t L = (size_t)N * N * H;
    std::memset(compact, 0, sizeof(float2) * 3 * g.sU);
    for (int q = 0; q < 3; ++q)
        for (int ix = 0; ix < g.NK; ++ix)
            for (int iy = 0; iy < g.NK; ++iy)
                for (int kz = 0; kz < g.NZ; ++kz) {
                    const int kx = ix <= g.kc ? ix : ix - g.NK, ky = iy <= g.kc ? iy : iy - g.NK;
                    const size_t src = q * L + ((size_t)((kx + N) % N) * N + (ky + N) % N) * H + kz;
                    compact[q * g.sU + ((size_t)ix * g.NK + iy) * g.NZp + kz] =
                        make_float2((float)full[2 * src], (float)full[2 * src + 1]);
                }
}

}  // namespace

static ens_status init_context(ens_ctx *ctx, const ens_member_desc *m, int n, const ens_hist_spec *h)
{
    ens_status s = ENS_OK;

    // member parameters
    std::vector<MemberDev> md(n);
    for (int i = 0; i < n; ++i) {
        const ens_member_desc &d = m[i];
        MemberDev &x = md[slot_of(ctx, i)];
        std::memset(&x, 0, sizeof x);
        x.nu = d.nu;
        x.eps_inj = std::exp(d.lambda) * d.eps_bar;
        x.klo2 = d.k_lo * d.k_lo;
        x.khi2 = d.k_hi * d.k_hi;
        // |k|^2 is an integer: k_lo <= |k| <= k_hi (1e-9 slack) as integer bounds
        x.band_lo2 = (int)std::ceil(x.klo2 - 1e-9);
        x.band_hi2 = (int)std::floor(x.khi2 + 1e-9);
        x.dt_fixed = d.dt > 0.0 ? d.dt : 0.0;
        x.cfl = d.cfl;
        x.dt_max = d.dt_max;
        x.rk = d.rk_order;
        x.N = d.N;
        x.group = ctx->member_group[i];
        x.index_in_group = ctx->member_local[i];
        x.seed = d.seed;
        x.init_energy = d.init_energy;
        const Geo &g = ctx->groups[x.group].geo;
        x.nblk = g.NK * g.NZp / g.tile_x;   // update-pass CTAs (>= sums-kernel CTAs)
        x.dt = x.dt_fixed;
    }
    cudaStream_t st = ctx->stream;
    int dev = 0;
    ENS_CUDA(ctx, cudaGetDevice(&dev));
    ENS_CUDA(ctx, cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, dev));
    ENS_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    ENS_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    ctx->aux.assign(ctx->groups.size(), nullptr);
    ctx->ev_join.assign(ctx->groups.size(), nullptr);
    for (size_t gi = 1; gi < ctx->groups.size(); ++gi) {
        ENS_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->aux[gi], cudaStreamNonBlocking));
        ENS_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_join[gi], cudaEventDisableTiming));
    }
    ENS_CUDA(ctx, cudaMemcpyAsync(ctx->md, md.data(), sizeof(MemberDev) * n, cudaMemcpyHostToDevice, st));
    ENS_CUDA(ctx, cudaMemsetAsync(ctx->partial, 0, sizeof(double) * n * ctx->partial_blocks * 4, st));
    const long long L = counts_len_of(h->qr_bins, h->tail_bins, h->grad_bins);
    ENS_CUDA(ctx, cudaMemsetAsync(ctx->counts, 0, sizeof(unsigned long long) * n * L, st));
    ENS_CUDA(ctx, cudaMemsetAsync(ctx->moments, 0, sizeof(double) * n * kNMom, st));
    // histogram edges and scalings
    HistDev &hd = ctx->hd;
    hd.nq = h->qr_bins;
    hd.nt = h->tail_bins;
    hd.counts_len = (int)L;
    const double q0 = h->eps_norm / (2.0 * h->nu_norm);
    hd.q_scale = (float)(1.0 / q0);
    hd.r_scale = (float)(1.0 / std::pow(q0, 1.5));
    hd.eps_scale = (float)(1.0 / h->eps_norm);
    hd.ens_scale = (float)(h->nu_norm / h->eps_norm);
    hd.q_lo = (float)(-h->q_lim);
    hd.q_inv_w = (float)(h->qr_bins / (2.0 * h->q_lim));
    hd.r_lo = (float)(-h->r_lim);
    hd.r_inv_w = (float)(h->qr_bins / (2.0 * h->r_lim));
    hd.t_lo = (float)h->tail_lo;
    hd.t_inv_w = (float)(h->tail_bins / (h->tail_hi - h->tail_lo));
    hd.edges_q = ctx->edges;
    hd.edges_r = ctx->edges + (h->qr_bins + 1);
    hd.edges_t = ctx->edges + 2 * (h->qr_bins + 1);
    hd.ng = h->grad_bins;
    hd.g_scale = (float)(1.0 / std::sqrt(q0));
    hd.g_lo = (float)(-h->grad_lim);
    hd.g_inv_w = h->grad_bins > 0 ? (float)(h->grad_bins / (2.0 * h->grad_lim)) : 0.f;
    hd.edges_g = hd.edges_t + h->tail_bins + 1;
    launch_edges(ctx->edges, ctx->edges + (h->qr_bins + 1), ctx->edges + 2 * (h->qr_bins + 1),
                 const_cast<float *>(hd.edges_g), h->qr_bins, h->tail_bins, h->grad_bins, h->q_lim, h->r_lim,
                 h->tail_lo, h->tail_hi, h->grad_lim, st);
    int smem_optin = 0;
    ENS_CUDA(ctx, cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    for (auto &gr : ctx->groups) {
        const size_t need = stats_smem(gr.geo.N, h->qr_bins, h->tail_bins, h->grad_bins);
        if (need > (size_t)smem_optin) {
            char buf[256];
            snprintf(buf, sizeof buf,
                     "histogram layout too large for the statistics pass at N = %d: %zu bytes of shared memory per "
                     "CTA, the device offers %d (fewer Q-R, tail or gradient bins)",
                     gr.geo.N, need, smem_optin);
            return fail(ctx, ENS_EINVAL, buf);
        }
        ENS_CUDA(ctx, prepare_kernels(gr.geo.N, h->qr_bins, h->tail_bins, h->grad_bins));
        const int per_sm = znl_ctas_per_sm(gr.geo.N);
        if (per_sm <= 0 || ctx->sms <= 0) return fail(ctx, ENS_ECUDA, "occupancy query of the z pass failed");
        gr.geo.z_ctas = per_sm * ctx->sms;
        gr.geo.sms = ctx->sms;
        launch_twiddles(const_cast<float2 *>(gr.geo.tw), gr.geo.N, st);
        ENS_CUDA(ctx, cudaMemsetAsync(gr.geo.U, 0, sizeof(float2) * 3 * gr.geo.sU * gr.geo.members, st));
        ENS_CUDA(ctx, cudaMemsetAsync(gr.geo.S, 0, sizeof(float2) * 3 * gr.geo.sU * gr.geo.members, st));
        launch_ic(gr.geo, ctx->md, st);
    }
    std::vector<PItem> items;   // kept until the synchronisation below
    if (ctx->pitems) {
        std::vector<Geo> geos;
        for (auto &gr : ctx->groups) geos.push_back(gr.geo);
        unsigned need[kPSlots][kPKinds];
        persist_items(geos, items, need);
        ENS_CUDA(ctx, persist_prepare());
        const int per_sm = persist_ctas_per_sm();
        ctx->persist_ctas = per_sm > 0 ? per_sm * ctx->sms : 0;
        ENS_CUDA(ctx, cudaMemcpyAsync(ctx->pitems, items.data(), sizeof(PItem) * items.size(),
                                      cudaMemcpyHostToDevice, st));
    }
    ENS_CUDA(ctx, cudaGetLastError());
    s = resum(ctx);
    if (s != ENS_OK) return s;
    ENS_CUDA(ctx, cudaStreamSynchronize(st));
    return ENS_OK;
}

extern "C" {

const char *ens_status_string(ens_status s)
{
    switch (s) {
    case ENS_OK: return "ok";
    case ENS_EINVAL: return "invalid argument";
    case ENS_ENOMEM: return "out of device memory";
    case ENS_ECUDA: return "CUDA error";
    case ENS_ENONFINITE: return "non-finite field";
    case ENS_ETIMEOUT: return "device wait timed out";
    case ENS_ESTATE: return "band energy vanished";
    case ENS_EUNSUPPORTED: return "unsupported grid size";
    }
    return "unknown status";
}

const char *ens_last_error(const ens_ctx *ctx)
{
    if (!ctx) return "null context";
    return ctx->err.empty() ? "" : ctx->err.c_str();
}

int ens_counts_len(const ens_hist_spec *h)
{
    return h ? (int)counts_len_of(h->qr_bins, h->tail_bins, h->grad_bins > 0 ? h->grad_bins : 0) : 0;
}

ens_status ens_query(const ens_member_desc *m, int n, const ens_hist_spec *h, size_t *bytes)
{
    std::string why;
    const ens_status s = validate(m, n, h, why);
    if (s != ENS_OK) return s;
    if (!bytes) return ENS_EINVAL;
    *bytes = carve(m, n, h, nullptr, nullptr);
    return ENS_OK;
}

ens_status ens_create(const ens_member_desc *m, int n, const ens_hist_spec *h, void *workspace, size_t ws_bytes,
                      void *stream, ens_ctx **out)
{
    if (!out) return ENS_EINVAL;
    *out = nullptr;
    std::string why;
    ens_status s = validate(m, n, h, why);
    if (s != ENS_OK) {
        fprintf(stderr, "ens_create: %s\n", why.c_str());
        return s;
    }
    ens_ctx *ctx = new ens_ctx();
    ctx->desc.assign(m, m + n);
    ctx->hist = *h;
    ctx->rk = m[0].rk_order;
    ctx->stream = (cudaStream_t)stream;
    const size_t need = carve(m, n, h, nullptr, nullptr);
    if (workspace) {
        if (ws_bytes < need) {
            fprintf(stderr, "ens_create: workspace of %zu bytes, %zu needed\n", ws_bytes, need);
            delete ctx;
            return ENS_ENOMEM;
        }
        ctx->workspace = workspace;
    } else {
        cudaError_t e = cudaMalloc(&ctx->workspace, need);
        if (e != cudaSuccess) {
            delete ctx;
            return e == cudaErrorMemoryAllocation ? ENS_ENOMEM : ENS_ECUDA;
        }
        ctx->owns = true;
    }
    ctx->ws_bytes = need;
    char *base = reinterpret_cast<char *>(
        (reinterpret_cast<uintptr_t>(ctx->workspace) + kAlign - 1) / kAlign * kAlign);
    carve(m, n, h, base, ctx);
    s = init_context(ctx, m, n, h);
    if (s != ENS_OK) {
        fprintf(stderr, "ens_create: %s\n", ctx->err.c_str());
        ens_destroy(ctx);
        return s;
    }
    *out = ctx;
    return ENS_OK;
}

ens_status ens_destroy(ens_ctx *ctx)
{
    if (!ctx) return ENS_EINVAL;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (auto st : ctx->aux)
        if (st) cudaStreamDestroy(st);
    for (auto ev : ctx->ev_join)
        if (ev) cudaEventDestroy(ev);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->copy_in) cudaStreamSynchronize(ctx->copy_in);
    if (ctx->copy_out) cudaStreamSynchronize(ctx->copy_out);
    if (ctx->copy_in) cudaStreamDestroy(ctx->copy_in);
    if (ctx->copy_out) cudaStreamDestroy(ctx->copy_out);
    if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
    for (auto ev : ctx->ev_in) cudaEventDestroy(ev);
    for (auto ev : ctx->ev_done) cudaEventDestroy(ev);
    if (ctx->owns && ctx->workspace) cudaFree(ctx->workspace);
    delete ctx;
    return ENS_OK;
}

int ens_members(const ens_ctx *ctx) { return ctx ? (int)ctx->desc.size() : 0; }
int ens_member_n(const ens_ctx *ctx, int i)
{
    return (ctx && i >= 0 && i < (int)ctx->desc.size()) ? ctx->desc[i].N : 0;
}
int ens_kernels_per_step(const ens_ctx *ctx)
{
    if (!ctx) return 0;
    if (ctx->persistent) return ctx->rk;   // one persistent launch per stage
    int per_stage = 1;   // the per-member stage reduction
    for (auto &gr : ctx->groups) per_stage += 5 + (gr.geo.fx_split == 1 ? 1 : 0);
    return ctx->rk * per_stage;
}

ens_status ens_step_sequential(ens_ctx *ctx, int nsteps)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (nsteps < 0) return fail(ctx, ENS_EINVAL, "nsteps < 0");
    for (int k = 0; k < nsteps; ++k) record_step_sequential(ctx, ctx->stream);
    ENS_CUDA(ctx, cudaGetLastError());
    return ENS_OK;
}

ens_status ens_step_nograph(ens_ctx *ctx, int nsteps)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (nsteps < 0) return fail(ctx, ENS_EINVAL, "nsteps < 0");
    Geo *armed = nullptr;   // ens_test_skip_copy: applies to this call's launches only
    if (ctx->skip_member >= 0) {
        armed = &ctx->groups[ctx->member_group[ctx->skip_member]].geo;
        armed->z_skip_member = ctx->member_local[ctx->skip_member];
        armed->z_skip_wait = ctx->skip_wait;
        ctx->skip_member = -1;
    }
    for (int k = 0; k < nsteps; ++k) record_step(ctx, ctx->stream);
    if (armed) armed->z_skip_member = -1;
    ENS_CUDA(ctx, cudaGetLastError());
    return ENS_OK;
}

ens_status ens_test_skip_copy(ens_ctx *ctx, int member, int wait_polls)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (member < 0 || member >= (int)ctx->desc.size() || wait_polls < 1 || wait_polls > (1 << 16)) {
        std::fprintf(stderr, "libens: ens_test_skip_copy: member out of range or wait_polls not in [1, 65536]\n");
        return ENS_EINVAL;
    }
    if (ctx->groups[ctx->member_group[member]].geo.z_mode == 1) {
        std::fprintf(stderr, "libens: ens_test_skip_copy: the member's group runs the z pass without bulk copies\n");
        return ENS_EINVAL;
    }
    ctx->skip_member = member;
    ctx->skip_wait = wait_polls;
    return ENS_OK;
}

ens_status ens_step(ens_ctx *ctx, int nsteps)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (nsteps < 0) return fail(ctx, ENS_EINVAL, "nsteps < 0");
    if (!ctx->graph) {
        cudaGraph_t graph;
        ENS_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        record_step(ctx, ctx->cap_stream);
        ENS_CUDA(ctx, cudaStreamEndCapture(ctx->cap_stream, &graph));
        cudaError_t e = cudaGraphInstantiate(&ctx->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(ctx, "cudaGraphInstantiate", e);
    }
    for (int k = 0; k < nsteps; ++k) ENS_CUDA(ctx, cudaGraphLaunch(ctx->graph, ctx->stream));
    return ENS_OK;
}

ens_status ens_step_host(ens_ctx *ctx, const void *host_in, void *host_out, size_t bytes, int chunk)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (!host_in || !host_out || bytes < ens_state_bytes(ctx) || chunk < 0)
        return fail(ctx, ENS_EINVAL, "ens_step_host: null buffer, state buffer too small or chunk < 0");
    if (!ctx->copy_in) {
        ENS_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_in, cudaStreamNonBlocking));
        ENS_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_out, cudaStreamNonBlocking));
        ENS_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming));
    }
    // chunk sizes per group: `chunk` members each, or (chunk = 0) sizes
    // growing by a factor 3 from one member up to a third of the group, the
    // middle in chunks of at most that, and the same sizes shrinking at the
    // end (M = 64: 1 3 9 19 19 9 3 1): the upload before the first compute and
    // the download after the last one are one member each, and each upload
    // (1/2.7 of its chunk's compute time per member at ~200 GB/s) lands while
    // the chunk before it computes; fewer chunks than equal eighths, so fewer
    // small launches
    std::vector<std::vector<int>> sched(ctx->groups.size());
    int nchunks = 0;
    for (size_t gi = 0; gi < ctx->groups.size(); ++gi) {
        const int M = ctx->groups[gi].geo.members;
        std::vector<int> &v = sched[gi];
        if (chunk > 0) {
            for (int k = 0; k < M; k += chunk) v.push_back(std::min(chunk, M - k));
        } else {
            const int cap = std::max(1, M / 3);
            std::vector<int> up;
            int used = 0;
            for (int sz = 1; sz <= cap && used + 2 * sz <= M; sz *= 3) {
                up.push_back(sz);
                used += 2 * sz;
            }
            int left = M - used;
            const int nmid = (left + cap - 1) / cap;
            v = up;
            for (int k = 0; k < nmid; ++k) {
                const int sz = left / (nmid - k);
                v.push_back(sz);
                left -= sz;
            }
            for (int k = (int)up.size() - 1; k >= 0; --k) v.push_back(up[k]);
        }
        nchunks += (int)v.size();
    }
    while ((int)ctx->ev_in.size() < nchunks) {
        cudaEvent_t a, b;
        ENS_CUDA(ctx, cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
        ENS_CUDA(ctx, cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
        ctx->ev_in.push_back(a);
        ctx->ev_done.push_back(b);
    }
    // the uploads overwrite U: earlier work of the context stream first
    ENS_CUDA(ctx, cudaEventRecord(ctx->ev_start, ctx->stream));
    ENS_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_in, ctx->ev_start, 0));
    const int PB = ctx->partial_blocks;
    const int nst = ctx->rk;
    const char *in = static_cast<const char *>(host_in);
    char *out = static_cast<char *>(host_out);
    size_t off = 0;
    int ci = 0;
    for (size_t gi = 0; gi < ctx->groups.size(); ++gi) {
        const Group &gr = ctx->groups[gi];
        const size_t per = sizeof(float2) * 3 * gr.geo.sU;
        int k0 = 0;
        for (const int cnt : sched[gi]) {
            const Geo g = member_range(gr.geo, k0, cnt);
            const size_t b = per * cnt;
            MemberDev *md = ctx->md + g.first;
            double *part = ctx->partial + (size_t)g.first * PB * 4;
            ENS_CUDA(ctx, cudaMemcpyAsync(g.U, in + off, b, cudaMemcpyHostToDevice, ctx->copy_in));
            ENS_CUDA(ctx, cudaEventRecord(ctx->ev_in[ci], ctx->copy_in));
            ENS_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_in[ci], 0));
            // energy sums of the uploaded state, as after ens_set_state
            ENS_CUDA(ctx, cudaMemsetAsync(part, 0, sizeof(double) * cnt * PB * 4, ctx->stream));
            launch_state_sums(g, ctx->md, ctx->stream);
            launch_finish(md, cnt, part, PB, 0, 0, 1, ctx->stream);
            for (int st = 0; st < nst; ++st) {
                const int last = st == nst - 1;
                record_group_stage(ctx, g, st, last, ctx->stream);
                launch_finish(md, cnt, part, PB, st, last, 0, ctx->stream);
            }
            ENS_CUDA(ctx, cudaEventRecord(ctx->ev_done[ci], ctx->stream));
            ENS_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_out, ctx->ev_done[ci], 0));
            ENS_CUDA(ctx, cudaMemcpyAsync(out + off, g.U, b, cudaMemcpyDeviceToHost, ctx->copy_out));
            off += b;
            k0 += cnt;
            ++ci;
        }
    }
    ENS_CUDA(ctx, cudaGetLastError());
    ENS_CUDA(ctx, cudaStreamSynchronize(ctx->copy_out));
    ENS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return ENS_OK;
}

ens_status ens_synchronize(ens_ctx *ctx)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    ENS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return ENS_OK;
}

ens_status ens_run_pass(ens_ctx *ctx, int pass, int stage)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (pass < 0 || pass > 4 || stage < 0 || stage >= ctx->rk) return fail(ctx, ENS_EINVAL, "bad pass/stage");
    const Pass kind[5] = {Pass::IX, Pass::IY, Pass::Z, Pass::FY, Pass::FX};
    for (auto &gr : ctx->groups) {
        const int mode = 0;
        const int arg = pass == 0 ? (stage > 0) : (pass == 1 ? 6 : 0);
        // the update pass is timed without writing the state back over U: it
        // targets S (not the last stage) so repeated profiling launches leave
        // the member state unchanged
        launch_pass(kind[pass], mode, gr.geo, ctx->md, nullptr, stage, 0, arg, ctx->stream);
    }
    ENS_CUDA(ctx, cudaGetLastError());
    return ENS_OK;
}

double ens_pass_bytes(const ens_ctx *ctx, int pass, int stage)
{
    if (!ctx) return 0.0;
    double total = 0.0;
    for (auto &gr : ctx->groups) {
        const Geo &g = gr.geo;
        const double c = 8.0;   // bytes per complex value
        const double st = (double)g.NK * g.NK * g.NZ * c;      // one state component
        const double a = (double)g.NK * g.N * g.NZ * c;        // one buffer-A field
        const double b = (double)g.N * g.N * g.NZ * c;         // one buffer-B field
        double bytes = 0.0;
        switch (pass) {
        case 0: bytes = 3 * st + 6 * a; break;
        case 1: bytes = 6 * a + 6 * b; break;
        case 2: bytes = 6 * b + 3 * b; break;
        case 3: bytes = 3 * b + 3 * a; break;
        case 4: bytes = 3 * a + (stage > 0 ? 2 : 1) * 3 * st + 3 * st; break;
        // statistics snapshot: 6 fields along x (u_i, i kx u_i from the 3
        // state comps), the 8 gradient components along y, then the z pass
        // that reads them for the invariants
        case 5: bytes = 3 * st + 6 * a + 6 * a + 8 * b + 8 * b; break;
        default: bytes = 0.0;
        }
        total += bytes * g.members;
    }
    return total;
}

ens_status ens_gradient_stats(ens_ctx *ctx, int accumulate)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    const int n = (int)ctx->desc.size();
    cudaStream_t st = ctx->stream;
    const long long L = ctx->hd.counts_len;
    if (!accumulate) {
        ENS_CUDA(ctx, cudaMemsetAsync(ctx->counts, 0, sizeof(unsigned long long) * n * L, st));
    }
    ENS_CUDA(ctx, cudaMemsetAsync(ctx->mom_partial, 0, sizeof(double) * n * ctx->mom_blocks * kNMom, st));
    for (auto &gr : ctx->groups) {
        const Geo &g = gr.geo;
        launch_pass(Pass::IX, 1, g, ctx->md, nullptr, 0, 0, 0, st);
        launch_pass(Pass::IY, kIYGrad, g, ctx->md, nullptr, 0, 0, 6, st);
        launch_pass(Pass::ZSTAT, 0, g, ctx->md, &ctx->hd, 0, 0, 0, st);
    }
    launch_finish_stats(ctx->mom_partial, ctx->mom_blocks, ctx->moments, n, accumulate, st);
    ENS_CUDA(ctx, cudaGetLastError());
    return ENS_OK;
}

ens_status ens_get_stats(ens_ctx *ctx, uint64_t *counts, double *moments)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    const int n = (int)ctx->desc.size();
    const long long L = ctx->hd.counts_len;
    std::vector<unsigned long long> c((size_t)n * L);
    std::vector<double> mo((size_t)n * kNMom);
    ENS_CUDA(ctx, cudaMemcpyAsync(c.data(), ctx->counts, sizeof(unsigned long long) * c.size(), cudaMemcpyDeviceToHost, ctx->stream));
    ENS_CUDA(ctx, cudaMemcpyAsync(mo.data(), ctx->moments, sizeof(double) * mo.size(), cudaMemcpyDeviceToHost, ctx->stream));
    ENS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < n; ++i) {
        const int sl = slot_of(ctx, i);
        if (counts) std::memcpy(counts + (size_t)i * L, c.data() + (size_t)sl * L, sizeof(uint64_t) * L);
        if (moments) std::memcpy(moments + (size_t)i * kNMom, mo.data() + (size_t)sl * kNMom, sizeof(double) * kNMom);
    }
    return ENS_OK;
}

ens_status ens_bin_check(ens_ctx *ctx, int axis, const float *values, int n, int *bins)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (axis < 0 || axis > 3 || n < 0 || (n > 0 && (!values || !bins)) || (axis == 3 && ctx->hd.ng <= 0))
        return fail(ctx, ENS_EINVAL, "ens_bin_check: axis 0..3 (3 needs grad_bins > 0), n >= 0, buffers");
    if (n == 0) return ENS_OK;
    float *dx = nullptr;
    int *db = nullptr;
    if (cudaMalloc(&dx, sizeof(float) * n) != cudaSuccess || cudaMalloc(&db, sizeof(int) * n) != cudaSuccess) {
        if (dx) cudaFree(dx);
        return fail(ctx, ENS_ENOMEM, "ens_bin_check: device buffers");
    }
    cudaError_t e = cudaMemcpyAsync(dx, values, sizeof(float) * n, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        launch_bin_check(ctx->hd, axis, dx, n, db, ctx->stream);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(bins, db, sizeof(int) * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(dx);
    cudaFree(db);
    ENS_CUDA(ctx, e);
    return ENS_OK;
}

static ens_status mixture_device(ens_ctx *ctx, int n, const double *d_lam, const unsigned long long *d_counts,
                                 const double *d_mom, const ens_hist_spec *h, const ens_weight_spec *w,
                                 const double *d_user, double *d_scratch, ens_mixture_out *out, cudaStream_t st)
{
    MixWeightArgs wa{};
    wa.kind = w->kind;
    wa.c = w->c;
    wa.Z = w->Z;
    wa.mu = w->mu;
    wa.sigma = w->sigma;
    wa.user = d_user;
    wa.renormalize = w->renormalize;
    MixPdfArgs pa{};
    pa.nq = h->qr_bins;
    pa.nt = h->tail_bins;
    pa.ng = h->grad_bins;
    pa.counts_len = (int)counts_len_of(h->qr_bins, h->tail_bins, h->grad_bins);
    pa.dq = 2.0 * h->q_lim / h->qr_bins;
    pa.dr = 2.0 * h->r_lim / h->qr_bins;
    pa.dt = (h->tail_hi - h->tail_lo) / h->tail_bins;
    pa.dg = h->grad_bins > 0 ? 2.0 * h->grad_lim / h->grad_bins : 0.0;
    const int nb = mix_pdf_len(pa);
    double *d_w = d_scratch, *d_cov = d_w + n, *d_pdf = d_cov + 1, *d_mm = d_pdf + nb, *d_rat = d_mm + kNMom;
    launch_mixture(d_lam, n, wa, d_counts, d_mom, pa, d_w, d_cov, d_pdf, d_mm, d_rat, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ctx ? cuda_fail(ctx, "mixture kernels", e) : ENS_ECUDA;
    std::vector<double> host((size_t)n + 1 + nb + kNMom + 5);
    e = cudaMemcpyAsync(host.data(), d_scratch, sizeof(double) * host.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ctx ? cuda_fail(ctx, "mixture copy", e) : ENS_ECUDA;
    const double *hw = host.data(), *hc = hw + n, *hp = hc + 1, *hm = hp + nb, *hr = hm + kNMom;
    if (out->weights) std::memcpy(out->weights, hw, sizeof(double) * n);
    out->covered = *hc;
    const int nq2 = h->qr_bins * h->qr_bins;
    if (out->pdf_qr) std::memcpy(out->pdf_qr, hp, sizeof(double) * nq2);
    if (out->pdf_eps) std::memcpy(out->pdf_eps, hp + nq2, sizeof(double) * h->tail_bins);
    if (out->pdf_ens) std::memcpy(out->pdf_ens, hp + nq2 + h->tail_bins, sizeof(double) * h->tail_bins);
    if (h->grad_bins > 0 && out->pdf_long)
        std::memcpy(out->pdf_long, hp + nq2 + 2 * h->tail_bins, sizeof(double) * h->grad_bins);
    if (h->grad_bins > 0 && out->pdf_trans)
        std::memcpy(out->pdf_trans, hp + nq2 + 2 * h->tail_bins + h->grad_bins, sizeof(double) * h->grad_bins);
    if (out->moments) std::memcpy(out->moments, hm, sizeof(double) * kNMom);
    for (int k = 0; k < 5; ++k) out->ratios[k] = hr[k];
    return ENS_OK;
}

static bool weight_spec_ok(const ens_weight_spec *w)
{
    if (!w) return false;
    switch (w->kind) {
    case ENS_W_GAUSS_PAPER: return w->c > 0.0 && w->Z >= 0.0;
    case ENS_W_TRUNC_GAUSS: return w->c > 0.0 && w->Z > 0.0;
    case ENS_W_GAUSS: return w->sigma > 0.0;
    case ENS_W_USER: return w->user != nullptr;
    }
    return false;
}

ens_status ens_mixture(ens_ctx *ctx, const ens_weight_spec *w, ens_mixture_out *out)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (!out || !weight_spec_ok(w)) return fail(ctx, ENS_EINVAL, "invalid weight specification");
    const int n = (int)ctx->desc.size();
    // lambdas and user weights in device slot order
    std::vector<double> lam(n), user(n, 0.0);
    for (int i = 0; i < n; ++i) {
        lam[slot_of(ctx, i)] = ctx->desc[i].lambda;
        if (w->kind == ENS_W_USER) user[slot_of(ctx, i)] = w->user[i];
    }
    double *d_lam = ctx->mix, *d_user = ctx->mix + n, *d_scr = ctx->mix + 2 * n;
    ENS_CUDA(ctx, cudaMemcpyAsync(d_lam, lam.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
    ENS_CUDA(ctx, cudaMemcpyAsync(d_user, user.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
    std::vector<double> wslot(n);
    ens_mixture_out tmp = *out;
    tmp.weights = wslot.data();
    s = mixture_device(ctx, n, d_lam, ctx->counts, ctx->moments, &ctx->hist, w, d_user, d_scr, &tmp, ctx->stream);
    if (s != ENS_OK) return s;
    double *keep = out->weights;
    *out = tmp;
    out->weights = keep;
    if (keep)
        for (int i = 0; i < n; ++i) keep[i] = wslot[slot_of(ctx, i)];
    return ENS_OK;
}

ens_status ens_mixture_host(int n, const double *lambdas, const uint64_t *counts, const double *moments,
                            const ens_hist_spec *h, const ens_weight_spec *w, ens_mixture_out *out, void *stream)
{
    if (n <= 0 || n > 1024 || !lambdas || !counts || !moments || !h || !out || !weight_spec_ok(w))
        return ENS_EINVAL;
    std::string why;
    if (validate_hist(h, why) != ENS_OK) return ENS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const long long L = counts_len_of(h->qr_bins, h->tail_bins, h->grad_bins);
    const size_t nd = (size_t)3 * n + 1 + L + kNMom + 8 + (size_t)n * kNMom;
    const size_t bytes = sizeof(double) * nd + sizeof(unsigned long long) * n * L;
    void *mem = nullptr;
    if (cudaMallocAsync(&mem, bytes, st) != cudaSuccess) return ENS_ENOMEM;
    double *d = (double *)mem;
    double *d_lam = d, *d_user = d + n, *d_mom = d + 2 * n, *d_scr = d_mom + (size_t)n * kNMom;
    unsigned long long *d_counts = reinterpret_cast<unsigned long long *>(d + nd);
    std::vector<double> user(n, 0.0);
    if (w->kind == ENS_W_USER) std::memcpy(user.data(), w->user, sizeof(double) * n);
    ens_status s = ENS_OK;
    if (cudaMemcpyAsync(d_lam, lambdas, sizeof(double) * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_user, user.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_mom, moments, sizeof(double) * n * kNMom, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_counts, counts, sizeof(uint64_t) * n * L, cudaMemcpyHostToDevice, st) != cudaSuccess)
        s = ENS_ECUDA;
    if (s == ENS_OK) s = mixture_device(nullptr, n, d_lam, d_counts, d_mom, h, w, d_user, d_scr, out, st);
    cudaFreeAsync(mem, st);
    cudaStreamSynchronize(st);
    return s;
}

ens_status ens_get_field(ens_ctx *ctx, int i, double *host)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (i < 0 || i >= (int)ctx->desc.size() || !host) return fail(ctx, ENS_EINVAL, "bad member or buffer");
    const Geo g = single(ctx, i);
    std::vector<float2> c((size_t)3 * g.sU);
    ENS_CUDA(ctx, cudaMemcpyAsync(c.data(), g.U, sizeof(float2) * c.size(), cudaMemcpyDeviceToHost, ctx->stream));
    ENS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    to_full(ctx, i, c.data(), host);
    return ENS_OK;
}

ens_status ens_set_field(ens_ctx *ctx, int i, const double *host)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (i < 0 || i >= (int)ctx->desc.size() || !host) return fail(ctx, ENS_EINVAL, "bad member or buffer");
    const Geo g = single(ctx, i);
    std::vector<float2> c((size_t)3 * g.sU);
    from_full(ctx, i, host, c.data());
    ENS_CUDA(ctx, cudaMemcpyAsync(g.U, c.data(), sizeof(float2) * c.size(), cudaMemcpyHostToDevice, ctx->stream));
    s = resum(ctx);
    if (s != ENS_OK) return s;
    ENS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return ENS_OK;
}

size_t ens_state_bytes(const ens_ctx *ctx)
{
    if (!ctx) return 0;
    size_t b = 0;
    for (auto &gr : ctx->groups) b += sizeof(float2) * 3 * gr.geo.sU * gr.geo.members;
    return b;
}

ens_status ens_get_state(ens_ctx *ctx, void *host, size_t bytes)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (!host || bytes < ens_state_bytes(ctx)) return fail(ctx, ENS_EINVAL, "state buffer too small");
    char *p = (char *)host;
    for (auto &gr : ctx->groups) {
        const size_t b = sizeof(float2) * 3 * gr.geo.sU * gr.geo.members;
        ENS_CUDA(ctx, cudaMemcpyAsync(p, gr.geo.U, b, cudaMemcpyDeviceToHost, ctx->stream));
        p += b;
    }
    ENS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return ENS_OK;
}

ens_status ens_set_state(ens_ctx *ctx, const void *host, size_t bytes)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (!host || bytes < ens_state_bytes(ctx)) return fail(ctx, ENS_EINVAL, "state buffer too small");
    const char *p = (const char *)host;
    for (auto &gr : ctx->groups) {
        const size_t b = sizeof(float2) * 3 * gr.geo.sU * gr.geo.members;
        ENS_CUDA(ctx, cudaMemcpyAsync(gr.geo.U, p, b, cudaMemcpyHostToDevice, ctx->stream));
        p += b;
    }
    return resum(ctx);
}

ens_status ens_get_velocity(ens_ctx *ctx, int i, double *host)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (i < 0 || i >= (int)ctx->desc.size() || !host) return fail(ctx, ENS_EINVAL, "bad member or buffer");
    const Geo g = single(ctx, i);
    launch_pass(Pass::IX, 0, g, ctx->md, nullptr, 0, 0, 0, ctx->stream);
    launch_pass(Pass::IY, 0, g, ctx->md, nullptr, 0, 0, 3, ctx->stream);
    launch_pass(Pass::Z, 3, g, ctx->md, nullptr, 0, 0, 0, ctx->stream);
    ENS_CUDA(ctx, cudaGetLastError());
    const size_t n3 = (size_t)g.N * g.N * g.N;
    std::vector<float> f(3 * n3);
    ENS_CUDA(ctx, cudaMemcpyAsync(f.data(), g.A, sizeof(float) * f.size(), cudaMemcpyDeviceToHost, ctx->stream));
    ENS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (size_t k = 0; k < f.size(); ++k) host[k] = f[k];
    return ENS_OK;
}

ens_status ens_set_velocity(ens_ctx *ctx, int i, const double *host)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (i < 0 || i >= (int)ctx->desc.size() || !host) return fail(ctx, ENS_EINVAL, "bad member or buffer");
    const Geo g = single(ctx, i);
    const size_t n3 = (size_t)g.N * g.N * g.N;
    std::vector<float> f(3 * n3);
    for (size_t k = 0; k < f.size(); ++k) f[k] = (float)host[k];
    ENS_CUDA(ctx, cudaMemcpyAsync(g.A, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice, ctx->stream));
    launch_pass(Pass::Z, 4, g, ctx->md, nullptr, 0, 0, 0, ctx->stream);
    launch_pass(Pass::FY, 0, g, ctx->md, nullptr, 0, 0, 0, ctx->stream);
    launch_pass(Pass::FX, 3, g, ctx->md, nullptr, 0, 0, 0, ctx->stream);
    ENS_CUDA(ctx, cudaGetLastError());
    s = resum(ctx);
    if (s != ENS_OK) return s;
    ENS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return ENS_OK;
}

ens_status ens_rhs(ens_ctx *ctx, int i, double *host)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (i < 0 || i >= (int)ctx->desc.size() || !host) return fail(ctx, ENS_EINVAL, "bad member or buffer");
    const Geo g = single(ctx, i);
    launch_pass(Pass::IX, 0, g, ctx->md, nullptr, 0, 0, 0, ctx->stream);
    launch_pass(Pass::IY, 0, g, ctx->md, nullptr, 0, 0, 6, ctx->stream);
    launch_pass(Pass::Z, 0, g, ctx->md, nullptr, 3, 0, 0, ctx->stream);   // max|u| into the spare slot 3
    launch_pass(Pass::FY, 0, g, ctx->md, nullptr, 0, 0, 0, ctx->stream);
    launch_pass(Pass::FX, 1, g, ctx->md, nullptr, 0, 0, 0, ctx->stream);
    ENS_CUDA(ctx, cudaGetLastError());
    std::vector<float2> c((size_t)3 * g.sU);
    ENS_CUDA(ctx, cudaMemcpyAsync(c.data(), g.S, sizeof(float2) * c.size(), cudaMemcpyDeviceToHost, ctx->stream));
    ENS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    to_full(ctx, i, c.data(), host);
    return ENS_OK;
}

ens_status ens_diagnostics(ens_ctx *ctx, ens_diag *out)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (!out) return fail(ctx, ENS_EINVAL, "null output");
    const int n = (int)ctx->desc.size();
    std::vector<MemberDev> md(n);
    ENS_CUDA(ctx, cudaMemcpyAsync(md.data(), ctx->md, sizeof(MemberDev) * n, cudaMemcpyDeviceToHost, ctx->stream));
    ENS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int any = 0;
    for (int i = 0; i < n; ++i) {
        const MemberDev &d = md[slot_of(ctx, i)];
        ens_diag &o = out[i];
        o.t = d.t;
        o.dt = d.dt;
        o.E = d.E;
        o.diss = d.diss;
        o.EB = d.EB;
        o.P = d.P;
        o.umax = d.umax;
        o.Rlambda = d.diss > 0 ? std::sqrt(20.0 * d.E * d.E / (3.0 * d.nu * d.diss)) : 0.0;
        o.kmeta = d.diss > 0 ? (d.N / 3.0) * std::pow(d.nu * d.nu * d.nu / d.diss, 0.25) : 0.0;
        o.steps = d.steps;
        o.flags = d.flags;
        o.reserved = 0;
        any |= d.flags;
    }
    // a member whose device wait gave up was left partly unprocessed, which
    // can also make it non-finite: the timeout is the cause and is reported first
    if (any & kFlagTimeout) return ENS_ETIMEOUT;
    if (any & kFlagNonFinite) return ENS_ENONFINITE;
    if (any & kFlagNoBandEnergy) return ENS_ESTATE;
    return ENS_OK;
}

}  // extern "C"

// ---- autotuner ------------------------------------------------------------

namespace {

void tuning_of(const ens_ctx *ctx, ens_tuning *t)
{
    std::memset(t, 0, sizeof *t);
    t->groups = (int)ctx->groups.size();
    t->parallel_groups = ctx->parallel_groups;
    t->persistent = ctx->persistent;
    for (size_t gi = 0; gi < ctx->groups.size() && gi < ENS_MAX_GROUPS; ++gi) {
        const Geo &g = ctx->groups[gi].geo;
        ens_group_tuning &o = t->group[gi];
        o.N = g.N;
        o.tile_x = g.tile_x;
        o.tile_y = g.tile_y;
        o.z_variant = g.z_mode;
        o.z_ctas_per_sm = ctx->sms > 0 ? g.z_ctas / ctx->sms : 0;
        o.plan_x = g.plan_x;
        o.fx_split = g.fx_split;
    }
}

ens_status tuning_valid(const ens_ctx *ctx, const ens_tuning *t, std::string &why)
{
    if (t->groups != (int)ctx->groups.size()) {
        why = "tuning describes a different number of grid-size groups";
        return ENS_EINVAL;
    }
    if (t->parallel_groups != 0 && t->parallel_groups != 1) {
        why = "parallel_groups must be 0 or 1";
        return ENS_EINVAL;
    }
    if (t->persistent != 0 && t->persistent != 1) {
        why = "persistent must be 0 or 1";
        return ENS_EINVAL;
    }
    if (t->persistent == 1 && (!ctx->pitems || ctx->persist_ctas <= 0)) {
        why = "the persistent stage kernel needs grid sizes among 128, 256 and 384";
        return ENS_EINVAL;
    }
    for (int gi = 0; gi < t->groups; ++gi) {
        const ens_group_tuning &o = t->group[gi];
        const int N = ctx->groups[gi].geo.N;
        if (o.N != N) {
            why = "tuning group " + std::to_string(gi) + " is for N = " + std::to_string(o.N) + ", not " +
                  std::to_string(N);
            return ENS_EINVAL;
        }
        if ((o.tile_x != 8 && o.tile_x != 16) || (o.tile_y != 8 && o.tile_y != 16)) {
            why = "column tiles must be 8 or 16";
            return ENS_EINVAL;
        }
        if (o.plan_x != 0 && !(o.plan_x == 1 && plan_variant_available(N))) {
            why = "plan_x must be 0, or 1 for N = 128, 256, 512";
            return ENS_EINVAL;
        }
        if (o.fx_split < 0 || o.fx_split > 2 || (o.fx_split == 2 && !fx_ws_available(N))) {
            why = "fx_split must be 0, 1, or 2 for N = 256";
            return ENS_EINVAL;
        }
        if (o.z_variant < 0 || o.z_variant > 2 || (o.z_variant == 2 && !zplan_variant_available(N))) {
            why = "z_variant must be 0, 1, or 2 for N = 256";
            return ENS_EINVAL;
        }
        const int occ = znl_ctas_per_sm(N, o.z_variant == 2 ? 1 : 0);
        if (o.z_ctas_per_sm < 1 || o.z_ctas_per_sm > occ) {
            why = "z_ctas_per_sm must lie in [1, " + std::to_string(occ) + "] for N = " + std::to_string(N);
            return ENS_EINVAL;
        }
    }
    return ENS_OK;
}

// MemberDev::nblk of every member (one int per struct, strided) from its
// group's current update-pass tile; synchronises
ens_status sync_nblk(ens_ctx *ctx)
{
    for (auto &gr : ctx->groups) {
        const Geo &g = gr.geo;
        // the persistent stage kernel runs the fused update pass on 16-column tiles
        const int nblk = ctx->persistent || g.fx_split == 2 ? g.NK * g.NZp / 16
                         : g.fx_split                     ? (int)((g.sU + kUpdChunk - 1) / kUpdChunk)
                                                          : g.NK * g.NZp / g.tile_x;
        std::vector<int> v(g.members, nblk);
        ENS_CUDA(ctx, cudaMemcpy2DAsync(&ctx->md[g.first].nblk, sizeof(MemberDev), v.data(), sizeof(int),
                                        sizeof(int), g.members, cudaMemcpyHostToDevice, ctx->stream));
    }
    ENS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return ENS_OK;
}

// Install a (validated) tuning: pass variants per group, the update pass's
// partial-sum count per member, and a fresh graph at the next ens_step.
ens_status apply_tuning(ens_ctx *ctx, const ens_tuning *t)
{
    ctx->parallel_groups = t->parallel_groups;
    ctx->persistent = t->persistent;
    for (int gi = 0; gi < t->groups; ++gi) {
        Geo &g = ctx->groups[gi].geo;
        const ens_group_tuning &o = t->group[gi];
        g.tile_x = o.tile_x;
        g.tile_y = o.tile_y;
        g.plan_x = o.plan_x;
        g.fx_split = o.fx_split;
        g.z_mode = o.z_variant;
        g.z_ctas = o.z_ctas_per_sm * ctx->sms;
    }
    const ens_status ns = sync_nblk(ctx);
    if (ns != ENS_OK) return ns;
    // slots a narrower tile wrote before must not leak into the reduction
    ENS_CUDA(ctx, cudaMemsetAsync(ctx->partial, 0,
                                  sizeof(double) * ctx->desc.size() * ctx->partial_blocks * 4, ctx->stream));
    ENS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    return ENS_OK;
}

}  // namespace

extern "C" {

ens_status ens_get_tuning(const ens_ctx *ctx, ens_tuning *out)
{
    if (!ctx || !out) return ENS_EINVAL;
    tuning_of(ctx, out);
    return ENS_OK;
}

ens_status ens_set_tuning(ens_ctx *ctx, const ens_tuning *t)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (!t) return fail(ctx, ENS_EINVAL, "null tuning");
    std::string why;
    if (tuning_valid(ctx, t, why) != ENS_OK) {
        ctx->err = why;   // not sticky: the context keeps its previous tuning
        return ENS_EINVAL;
    }
    return apply_tuning(ctx, t);
}

ens_status ens_autotune(ens_ctx *ctx, int steps, ens_tuning *out)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (steps < 1) return fail(ctx, ENS_EINVAL, "autotune needs at least one timed step per trial");
    const int n = (int)ctx->desc.size();
    cudaStream_t st = ctx->stream;
    // snapshot of the member state: the spectral fields U (S is stage
    // scratch, rewritten before it is read) and the per-member run state
    size_t bytes = sizeof(MemberDev) * n;
    for (auto &gr : ctx->groups) bytes += sizeof(float2) * 3 * gr.geo.sU * gr.geo.members;
    char *snap = nullptr;
    if (cudaMallocAsync(&snap, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        ctx->err = "autotune: no device memory for the state snapshot (" + std::to_string(bytes) + " bytes)";
        return ENS_ENOMEM;
    }
    auto copy_state = [&](bool save) -> cudaError_t {
        size_t off = 0;
        cudaError_t e = cudaSuccess;
        for (auto &gr : ctx->groups) {
            const size_t b = sizeof(float2) * 3 * gr.geo.sU * gr.geo.members;
            e = save ? cudaMemcpyAsync(snap + off, gr.geo.U, b, cudaMemcpyDeviceToDevice, st)
                     : cudaMemcpyAsync(gr.geo.U, snap + off, b, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return e;
            off += b;
        }
        return save ? cudaMemcpyAsync(snap + off, ctx->md, sizeof(MemberDev) * n, cudaMemcpyDeviceToDevice, st)
                    : cudaMemcpyAsync(ctx->md, snap + off, sizeof(MemberDev) * n, cudaMemcpyDeviceToDevice, st);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ens_tuning best, cand;
    tuning_of(ctx, &best);
    const ens_tuning start = best;
    double best_ms = 0.0;
    int trials = 0;
    ens_status rs = ENS_OK;
    auto fail_cuda = [&](const char *what, cudaError_t e) {
        rs = cuda_fail(ctx, what, e);
        return -1.0;
    };
    // one trial: install, restore the snapshot, one untimed step, then the
    // mean of `steps` graph launches between two events
    // (the snapshot holds the per-member partial-sum counts of the starting
    // tuning, so the state is restored first and the tuning installed after)
    auto trial = [&](const ens_tuning &t) -> double {
        cudaError_t e = copy_state(false);
        if (e != cudaSuccess) return fail_cuda("autotune restore", e);
        if (apply_tuning(ctx, &t) != ENS_OK) {
            rs = ctx->sticky != ENS_OK ? ctx->sticky : ENS_ECUDA;
            return -1.0;
        }
        if (ens_step(ctx, 1) != ENS_OK) {
            rs = ctx->sticky;
            return -1.0;
        }
        if ((e = cudaEventRecord(e0, st)) != cudaSuccess) return fail_cuda("cudaEventRecord", e);
        if (ens_step(ctx, steps) != ENS_OK) {
            rs = ctx->sticky;
            return -1.0;
        }
        if ((e = cudaEventRecord(e1, st)) != cudaSuccess) return fail_cuda("cudaEventRecord", e);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return fail_cuda("cudaEventSynchronize", e);
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) return fail_cuda("cudaEventElapsedTime", e);
        ++trials;
        return ms / steps;
    };
    // a candidate replaces the incumbent only if it is faster by more than
    // the timing noise of one trial
    constexpr double kMargin = 0.01;
    auto consider = [&](const ens_tuning &t) -> bool {
        const double ms = trial(t);
        if (ms < 0.0) return false;
        if (ms < best_ms * (1.0 - kMargin)) {
            best = t;
            best_ms = ms;
        }
        return true;
    };
    cudaError_t e = copy_state(true);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        rs = cuda_fail(ctx, "autotune setup", e);
    } else {
        best_ms = trial(best);
        if (best_ms < 0.0) rs = rs == ENS_OK ? ENS_ECUDA : rs;
    }
    // coordinate descent over the knobs in two sweeps: parallel or serial
    // grid-size groups first (the groups' own knobs rank differently under
    // the two), then group by group; in the first sweep a group's gain is
    // judged against a step whose later groups are still untuned (a smaller
    // relative gain than once they are tuned)
    for (int sweep = 0; sweep < 2; ++sweep)
    for (int gi = -1; rs == ENS_OK && gi < best.groups; ++gi) {
        if (gi < 0) {
            if (sweep == 1) {
                // the incumbent's time afresh: the time it won with is biased
                // low (the fastest of several noisy trials)
                const double ms = trial(best);
                if (ms < 0.0) break;
                best_ms = ms;
            }
            if (best.groups > 1) {
                cand = best;
                cand.parallel_groups = 1 - best.parallel_groups;
                if (!consider(cand)) break;
            }
            continue;
        }
        const int N = best.group[gi].N;
        if (plan_variant_available(N)) {
            cand = best;
            cand.group[gi].plan_x = 1 - best.group[gi].plan_x;
            if (!consider(cand)) break;
        }
        for (int tile : {16, 8}) {
            cand = best;
            if (cand.group[gi].tile_x == tile) continue;
            cand.group[gi].tile_x = tile;
            if (!consider(cand)) break;
        }
        for (int tile : {16, 8}) {
            if (rs != ENS_OK) break;
            cand = best;
            if (cand.group[gi].tile_y == tile) continue;
            cand.group[gi].tile_y = tile;
            if (!consider(cand)) break;
        }
        const int occ = znl_ctas_per_sm(N);
        for (int c = 1; rs == ENS_OK && c <= occ; ++c) {
            cand = best;
            if (cand.group[gi].z_variant == 0 && cand.group[gi].z_ctas_per_sm == c) continue;
            cand.group[gi].z_variant = 0;
            cand.group[gi].z_ctas_per_sm = c;
            if (!consider(cand)) break;
        }
        if (zplan_variant_available(N)) {
            const int occ2 = znl_ctas_per_sm(N, 1);
            for (int c = 1; rs == ENS_OK && c <= occ2; ++c) {
                cand = best;
                if (cand.group[gi].z_variant == 2 && cand.group[gi].z_ctas_per_sm == c) continue;
                cand.group[gi].z_variant = 2;
                cand.group[gi].z_ctas_per_sm = c;
                if (!consider(cand)) break;
            }
        }
        if (rs == ENS_OK && best.group[gi].z_variant != 1) {
            cand = best;
            cand.group[gi].z_variant = 1;
            consider(cand);
        }
        for (int fx = 0; rs == ENS_OK && fx <= 2; ++fx) {
            if (fx == best.group[gi].fx_split || (fx == 2 && !fx_ws_available(N))) continue;
            cand = best;
            cand.group[gi].fx_split = fx;
            consider(cand);
        }
    }
    if (rs == ENS_OK && ctx->pitems && ctx->persist_ctas > 0) {
        cand = best;
        cand.persistent = 1;
        consider(cand);
    }
    // install the winner (or, after an error, the starting tuning) and put
    // the state back as it was
    const ens_tuning &fin = rs == ENS_OK ? best : start;
    if (ctx->sticky == ENS_OK) {
        e = copy_state(false);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess && rs == ENS_OK) rs = cuda_fail(ctx, "autotune restore", e);
        if (e == cudaSuccess) apply_tuning(ctx, &fin);
    }
    cudaFreeAsync(snap, st);
    cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) {
        *out = fin;
        out->ms_per_step = rs == ENS_OK ? best_ms : 0.0;
        out->trials = trials;
    }
    return rs;
}

}  // extern "C"

// ---- checkpoint / resume ------------------------------------------------------

namespace {

constexpr char kCkptMagic[8] = {'E', 'N', 'S', 'C', 'K', 'P', 'T', '1'};

struct CkptHeader {
    char magic[8];
    uint32_t version, members, rk, counts_len;
    uint64_t state_bytes, md_bytes, payload_hash;
    ens_hist_spec hist;
};

// FNV-1a over the payload, to refuse a truncated or altered file
uint64_t fnv1a(uint64_t h, const void *data, size_t n)
{
    const unsigned char *p = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

bool same_desc(const ens_member_desc &a, const ens_member_desc &b)
{
    return a.N == b.N && a.rk_order == b.rk_order && a.nu == b.nu && a.lambda == b.lambda &&
           a.eps_bar == b.eps_bar && a.k_lo == b.k_lo && a.k_hi == b.k_hi && a.dt == b.dt && a.cfl == b.cfl &&
           a.dt_max == b.dt_max && a.seed == b.seed && a.init_energy == b.init_energy;
}

bool same_hist(const ens_hist_spec &a, const ens_hist_spec &b)
{
    return a.qr_bins == b.qr_bins && a.q_lim == b.q_lim && a.r_lim == b.r_lim && a.tail_bins == b.tail_bins &&
           a.tail_lo == b.tail_lo && a.tail_hi == b.tail_hi && a.eps_norm == b.eps_norm && a.nu_norm == b.nu_norm &&
           a.grad_bins == b.grad_bins && (a.grad_bins == 0 || a.grad_lim == b.grad_lim);
}

}  // namespace

extern "C" {

ens_status ens_set_timestep(ens_ctx *ctx, int member, double dt, double cfl, double dt_max)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (member < 0 || member >= (int)ctx->desc.size() || !std::isfinite(dt) || !std::isfinite(cfl) ||
        !std::isfinite(dt_max) || (!(dt > 0.0) && !(cfl > 0.0))) {
        ctx->err = "ens_set_timestep: bad member or time-step rule";   // not sticky
        return ENS_EINVAL;
    }
    MemberDev *d = ctx->md + slot_of(ctx, member);
    const double v[3] = {dt > 0.0 ? dt : 0.0, cfl, dt_max};   // dt_fixed, cfl, dt_max are adjacent
    static_assert(offsetof(MemberDev, cfl) == offsetof(MemberDev, dt_fixed) + sizeof(double) &&
                      offsetof(MemberDev, dt_max) == offsetof(MemberDev, cfl) + sizeof(double),
                  "time-step fields must be contiguous");
    ENS_CUDA(ctx, cudaMemcpyAsync(&d->dt_fixed, v, sizeof v, cudaMemcpyHostToDevice, ctx->stream));
    ENS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return ENS_OK;
}

ens_status ens_save(ens_ctx *ctx, const char *path)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (!path) return fail(ctx, ENS_EINVAL, "null path");
    const int n = (int)ctx->desc.size();
    const size_t L = (size_t)counts_len_of(ctx->hist.qr_bins, ctx->hist.tail_bins, ctx->hist.grad_bins);
    const size_t sb = ens_state_bytes(ctx), mb = sizeof(MemberDev) * n;
    std::vector<char> state(sb), md(mb);
    std::vector<unsigned long long> counts(n * L);
    std::vector<double> mom((size_t)n * kNMom);
    s = ens_get_state(ctx, state.data(), sb);
    if (s != ENS_OK) return s;
    ENS_CUDA(ctx, cudaMemcpyAsync(md.data(), ctx->md, mb, cudaMemcpyDeviceToHost, ctx->stream));
    ENS_CUDA(ctx, cudaMemcpyAsync(counts.data(), ctx->counts, sizeof(unsigned long long) * counts.size(),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    ENS_CUDA(ctx, cudaMemcpyAsync(mom.data(), ctx->moments, sizeof(double) * mom.size(), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    ENS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    CkptHeader h{};
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = 1;
    h.members = (uint32_t)n;
    h.rk = (uint32_t)ctx->rk;
    h.counts_len = (uint32_t)L;
    h.state_bytes = sb;
    h.md_bytes = mb;
    h.hist = ctx->hist;
    uint64_t hash = 0xcbf29ce484222325ull;
    hash = fnv1a(hash, ctx->desc.data(), sizeof(ens_member_desc) * n);
    hash = fnv1a(hash, state.data(), sb);
    hash = fnv1a(hash, md.data(), mb);
    hash = fnv1a(hash, counts.data(), sizeof(unsigned long long) * counts.size());
    hash = fnv1a(hash, mom.data(), sizeof(double) * mom.size());
    h.payload_hash = hash;
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return fail(ctx, ENS_EINVAL, std::string("cannot open ") + tmp + " for writing");
    bool ok = std::fwrite(&h, sizeof h, 1, f) == 1 &&
              std::fwrite(ctx->desc.data(), sizeof(ens_member_desc), n, f) == (size_t)n &&
              std::fwrite(state.data(), 1, sb, f) == sb && std::fwrite(md.data(), 1, mb, f) == mb &&
              std::fwrite(counts.data(), sizeof(unsigned long long), counts.size(), f) == counts.size() &&
              std::fwrite(mom.data(), sizeof(double), mom.size(), f) == mom.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return fail(ctx, ENS_EINVAL, std::string("writing the checkpoint ") + path + " failed");
    }
    return ENS_OK;
}

ens_status ens_load(ens_ctx *ctx, const char *path)
{
    ens_status s = check(ctx);
    if (s != ENS_OK) return s;
    if (!path) return fail(ctx, ENS_EINVAL, "null path");
    auto refuse = [&](const std::string &why) {
        ctx->err = std::string("ens_load: ") + path + ": " + why;   // not sticky: the state is untouched
        return ENS_EINVAL;
    };
    FILE *f = std::fopen(path, "rb");
    if (!f) return refuse("cannot open");
    const int n = (int)ctx->desc.size();
    const size_t L = (size_t)counts_len_of(ctx->hist.qr_bins, ctx->hist.tail_bins, ctx->hist.grad_bins);
    const size_t sb = ens_state_bytes(ctx), mb = sizeof(MemberDev) * n;
    CkptHeader h{};
    std::vector<ens_member_desc> desc(n);
    std::vector<char> state(sb), md(mb);
    std::vector<unsigned long long> counts(n * L);
    std::vector<double> mom((size_t)n * kNMom);
    bool ok = std::fread(&h, sizeof h, 1, f) == 1 && std::memcmp(h.magic, kCkptMagic, 8) == 0 && h.version == 1;
    if (ok) ok = h.members == (uint32_t)n && h.rk == (uint32_t)ctx->rk && h.counts_len == (uint32_t)L &&
                 h.state_bytes == sb && h.md_bytes == mb && same_hist(h.hist, ctx->hist);
    if (!ok) {
        std::fclose(f);
        return refuse("not a checkpoint of an ensemble with these members and histograms");
    }
    ok = std::fread(desc.data(), sizeof(ens_member_desc), n, f) == (size_t)n &&
         std::fread(state.data(), 1, sb, f) == sb && std::fread(md.data(), 1, mb, f) == mb &&
         std::fread(counts.data(), sizeof(unsigned long long), counts.size(), f) == counts.size() &&
         std::fread(mom.data(), sizeof(double), mom.size(), f) == mom.size();
    std::fclose(f);
    if (!ok) return refuse("truncated");
    for (int i = 0; i < n; ++i)
        if (!same_desc(desc[i], ctx->desc[i])) return refuse("member " + std::to_string(i) + " differs");
    uint64_t hash = 0xcbf29ce484222325ull;
    hash = fnv1a(hash, desc.data(), sizeof(ens_member_desc) * n);
    hash = fnv1a(hash, state.data(), sb);
    hash = fnv1a(hash, md.data(), mb);
    hash = fnv1a(hash, counts.data(), sizeof(unsigned long long) * counts.size());
    hash = fnv1a(hash, mom.data(), sizeof(double) * mom.size());
    if (hash != h.payload_hash) return refuse("checksum mismatch");
    // the member run state, spectral state and statistics as saved; the
    // partial-sum counts follow this context's tuning
    const char *p = state.data();
    for (auto &gr : ctx->groups) {
        const size_t b = sizeof(float2) * 3 * gr.geo.sU * gr.geo.members;
        ENS_CUDA(ctx, cudaMemcpyAsync(gr.geo.U, p, b, cudaMemcpyHostToDevice, ctx->stream));
        p += b;
    }
    ENS_CUDA(ctx, cudaMemcpyAsync(ctx->md, md.data(), mb, cudaMemcpyHostToDevice, ctx->stream));
    ENS_CUDA(ctx, cudaMemcpyAsync(ctx->counts, counts.data(), sizeof(unsigned long long) * counts.size(),
                                  cudaMemcpyHostToDevice, ctx->stream));
    ENS_CUDA(ctx, cudaMemcpyAsync(ctx->moments, mom.data(), sizeof(double) * mom.size(), cudaMemcpyHostToDevice,
                                  ctx->stream));
    return sync_nblk(ctx);
}

}  // extern "C"
