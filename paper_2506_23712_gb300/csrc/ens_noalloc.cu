// ens_mixture_host_noalloc: the lambda mixture of host-side member
// statistics, for callers that must not allocate device memory.
//
// ens_mixture_host allocates temporary device memory for its inputs and
// outputs.  Some callers cannot do that: a process whose device memory is
// entirely reserved by another allocator (for example a framework's caching
// allocator that has claimed the GPU), or an application that budgets every
// device byte up front.  This entry point runs the same mixture kernels on a
// fixed scratch array that is part of the library image instead.
//
// The scratch is one file-scope __device__ array of kScratchBytes (about
// 4.3 MB), present on every GPU that loads the library until the process
// exits.  In host code its name is only a host-side stand-in, so the device
// address is looked up with cudaGetSymbolAddress, once per device, on the
// first call made while that device is current.
#include "../../include/ens.h"
#include "ens_launch.h"

#include <cstdio>
#include <mutex>

using namespace ens;

namespace {

constexpr int kMaxMembers = ENS_NOALLOC_MAX_MEMBERS;
constexpr int kMaxCounts = ENS_NOALLOC_MAX_COUNTS;
constexpr int kMaxDevices = 64;

// doubles: lambdas, user weights, moments, then the results (weights,
// covered mass, PDFs, mixed moments, ratios); counts follow as uint64
constexpr size_t kDoubles = (size_t)2 * kMaxMembers + (size_t)kMaxMembers * kNMom + kMaxMembers + 1 +
                            kMaxCounts + kNMom + 8;
constexpr size_t kDoublesPadded = (kDoubles + 31) / 32 * 32;
constexpr size_t kScratchBytes = sizeof(double) * kDoublesPadded +
                                 sizeof(unsigned long long) * (size_t)kMaxMembers * kMaxCounts;

__device__ __align__(256) unsigned char g_mixture_scratch[kScratchBytes];

std::mutex g_lock;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up once).
ens_status scratch_address(void **addr)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ENS_ECUDA;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_mixture_scratch);
        if (e != cudaSuccess) {
            fprintf(stderr, "ens_mixture_host_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
            return ENS_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *addr = g_scratch_addr[dev];
    return ENS_OK;
}

bool spec_ok(const ens_weight_spec *w)
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

}  // namespace

extern "C" ens_status ens_mixture_host_noalloc(int n, const double *lambdas, const uint64_t *counts,
                                               const double *moments, const ens_hist_spec *h,
                                               const ens_weight_spec *w, ens_mixture_out *out, void *stream)
{
    if (n <= 0 || !lambdas || !counts || !moments || !h || !out || !spec_ok(w)) return ENS_EINVAL;
    if (h->qr_bins < 1 || h->tail_bins < 1 || !(h->q_lim > 0) || !(h->r_lim > 0) || !(h->tail_hi > h->tail_lo))
        return ENS_EINVAL;
    if (h->grad_bins < 0 || (h->grad_bins > 0 && !(h->grad_lim > 0))) return ENS_EINVAL;
    const long long L = counts_len_of(h->qr_bins, h->tail_bins, h->grad_bins);
    if (n > kMaxMembers || L > kMaxCounts) {
        fprintf(stderr,
                "ens_mixture_host_noalloc: %d members x %lld counts exceed the fixed scratch "
                "(at most %d members and %d counts per member); use ens_mixture_host\n",
                n, L, kMaxMembers, kMaxCounts);
        return ENS_EINVAL;
    }
    void *base = nullptr;
    ens_status s = scratch_address(&base);
    if (s != ENS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    double *d = static_cast<double *>(base);
    double *d_lam = d, *d_user = d + kMaxMembers, *d_mom = d + 2 * kMaxMembers;
    double *d_w = d_mom + (size_t)kMaxMembers * kNMom, *d_cov = d_w + kMaxMembers, *d_pdf = d_cov + 1;
    double *d_mm = d_pdf + kMaxCounts, *d_rat = d_mm + kNMom;
    unsigned long long *d_counts = reinterpret_cast<unsigned long long *>(d + kDoublesPadded);

    // The scratch keeps whatever the previous call left.  Nothing has to
    // start at zero: every input slot the kernels read is copied in below,
    // and every output slot is written by the kernels before it is copied
    // back.
    cudaError_t e = cudaMemcpyAsync(d_lam, lambdas, sizeof(double) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && w->kind == ENS_W_USER)
        e = cudaMemcpyAsync(d_user, w->user, sizeof(double) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_mom, moments, sizeof(double) * n * kNMom, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_counts, counts, sizeof(uint64_t) * n * L, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return ENS_ECUDA;

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
    pa.counts_len = (int)L;
    pa.dq = 2.0 * h->q_lim / h->qr_bins;
    pa.dr = 2.0 * h->r_lim / h->qr_bins;
    pa.dt = (h->tail_hi - h->tail_lo) / h->tail_bins;
    pa.dg = h->grad_bins > 0 ? 2.0 * h->grad_lim / h->grad_bins : 0.0;
    launch_mixture(d_lam, n, wa, d_counts, d_mom, pa, d_w, d_cov, d_pdf, d_mm, d_rat, st);
    if (cudaGetLastError() != cudaSuccess) return ENS_ECUDA;

    // results straight into the caller's host buffers (no staging copy)
    const int nq2 = h->qr_bins * h->qr_bins;
    double ratios[5];
    if (out->weights) e = cudaMemcpyAsync(out->weights, d_w, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&out->covered, d_cov, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && out->pdf_qr)
        e = cudaMemcpyAsync(out->pdf_qr, d_pdf, sizeof(double) * nq2, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && out->pdf_eps)
        e = cudaMemcpyAsync(out->pdf_eps, d_pdf + nq2, sizeof(double) * h->tail_bins, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && out->pdf_ens)
        e = cudaMemcpyAsync(out->pdf_ens, d_pdf + nq2 + h->tail_bins, sizeof(double) * h->tail_bins,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && h->grad_bins > 0 && out->pdf_long)
        e = cudaMemcpyAsync(out->pdf_long, d_pdf + nq2 + 2 * h->tail_bins, sizeof(double) * h->grad_bins,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && h->grad_bins > 0 && out->pdf_trans)
        e = cudaMemcpyAsync(out->pdf_trans, d_pdf + nq2 + 2 * h->tail_bins + h->grad_bins,
                            sizeof(double) * h->grad_bins, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && out->moments)
        e = cudaMemcpyAsync(out->moments, d_mm, sizeof(double) * kNMom, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ratios, d_rat, sizeof(double) * 5, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ENS_ECUDA;
    for (int k = 0; k < 5; ++k) out->ratios[k] = ratios[k];
    return ENS_OK;
}
