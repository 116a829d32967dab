// Event ordering: validate the list-mode events and sort them by
// (subset, angle, energy class, position bin) with two stable counting-sort
// passes.  Subsets are formed from detector angles (paper Section 2.2):
// subset i holds the angles a with a mod N_s == i, so after sorting every
// subset, and every angle within it, is a contiguous range of model rows.
// Within an angle the events below the photopeak class (E < E0 (1 - f_E / 2),
// the lower half-maximum of the photopeak) come first, then those in it, each
// class ordered by position: a tile of consecutive events then needs a
// narrow strip of scatter pixels, and its events share an energy class, so
// that the path sum's energy cut (which drops the backscatter paths of
// photopeak events) drops them for whole warps alike.  Both passes are
// stable, so the order is a deterministic function of the input.
#include "lmosem_internal.cuh"

namespace lmosem {

namespace {

constexpr int kSortThreads = 256;
constexpr int kUBins = 512;
constexpr int kScanBlock = 1024;

__global__ void k_check_events(const int32_t* __restrict__ a, const float* __restrict__ u,
                               const float* __restrict__ e, int64_t n, int n_angles, float half,
                               float elo, float ehi, int* __restrict__ bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int ai = a[i];
    float ui = u[i], ei = e[i];
    bool ok = ai >= 0 && ai < n_angles && fabsf(ui) <= half && ei >= elo && ei <= ehi;
    if (!ok) atomicAdd(bad, 1);
}

// realisation of event (or sorted row) i: the last r with off[r] <= i
__device__ __forceinline__ int realisation_of(const int64_t* off, int n_real, int64_t i) {
    int lo = 0, hi = n_real - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// digit of the event at original index i
struct Digit {
    int mode;  // 0: (energy class, position bin), 1: subset-major angle slot, 2: realisation
    const int32_t* a;
    const float* u;
    float half;
    int n_subsets, group;
    const int64_t* off;
    int n_real;
    const float* e;
    float e_class;  // lower edge of the photopeak class
    __device__ int operator()(int64_t i) const {
        if (mode == 0) {
            int b = (int)floorf((u[i] + half) * ((float)kUBins / (2.0f * half)));
            return min(max(b, 0), kUBins - 1) + (e[i] >= e_class ? kUBins : 0);
        }
        if (mode == 2) return realisation_of(off, n_real, i);
        int ai = a[i];
        return (ai % n_subsets) * group + ai / n_subsets;
    }
};

// events per (realisation, angle) of the sorted rows
__global__ void k_rs_hist(const int32_t* __restrict__ a_s, int64_t n, const int64_t* __restrict__ off,
                          int n_real, int n_angles, int32_t* __restrict__ cnt) {
    int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    int r = off ? realisation_of(off, n_real, row) : 0;
    atomicAdd(&cnt[(size_t)r * n_angles + a_s[row]], 1);
}

// per-block digit histograms, digit-major: H[d * nblk + b]
__global__ void k_hist(Digit dg, const int32_t* __restrict__ perm, int64_t n, int ndig,
                       int32_t* __restrict__ H) {
    extern __shared__ int32_t sh[];
    int nblk = gridDim.x;
    for (int d = threadIdx.x; d < ndig; d += blockDim.x) sh[d] = 0;
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&sh[dg(perm ? perm[i] : i)], 1);
    __syncthreads();
    for (int d = threadIdx.x; d < ndig; d += blockDim.x) H[(size_t)d * nblk + blockIdx.x] = sh[d];
}

// exclusive scan, three phases
__global__ void k_scan_local(int32_t* __restrict__ x, int64_t n, int32_t* __restrict__ tot) {
    __shared__ int32_t s[kScanBlock];
    int64_t base = (int64_t)blockIdx.x * kScanBlock * 4;
    int t = threadIdx.x;
    int32_t v[4], run = 0;
    for (int k = 0; k < 4; ++k) {
        int64_t i = base + (int64_t)t * 4 + k;
        v[k] = i < n ? x[i] : 0;
        run += v[k];
    }
    s[t] = run;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {
        int32_t add = t >= off ? s[t - off] : 0;
        __syncthreads();
        s[t] += add;
        __syncthreads();
    }
    int32_t ex = s[t] - run;
    for (int k = 0; k < 4; ++k) {
        int64_t i = base + (int64_t)t * 4 + k;
        if (i < n) x[i] = ex;
        ex += v[k];
    }
    if (t == kScanBlock - 1) tot[blockIdx.x] = s[t];
}

__global__ void k_scan_totals(int32_t* __restrict__ tot, int n) {
    __shared__ int32_t s[kScanBlock];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += kScanBlock) {
        int i = base + threadIdx.x;
        int32_t v = i < n ? tot[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < kScanBlock; off <<= 1) {
            int32_t add = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
            __syncthreads();
            s[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < n) tot[i] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) carry += s[kScanBlock - 1];
        __syncthreads();
    }
}

__global__ void k_scan_add(int32_t* __restrict__ x, int64_t n, const int32_t* __restrict__ tot) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += tot[i / (kScanBlock * 4)];
}

// stable scatter: rank inside the block from warp match masks and per-warp
// digit counts
__global__ void k_scatter(Digit dg, const int32_t* __restrict__ perm_in, int64_t n, int ndig,
                          const int32_t* __restrict__ O, int32_t* __restrict__ perm_out) {
    extern __shared__ int32_t wc[];  // [warps][ndig]
    const int nw = kSortThreads / 32;
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < nw * ndig; k += blockDim.x) wc[k] = 0;
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = i < n;
    int32_t src = valid ? (perm_in ? perm_in[i] : (int32_t)i) : 0;
    int d = valid ? dg(src) : -1 - lane;  // invalid lanes never match a digit
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int lrank = __popc(peers & ((1u << lane) - 1u));
    if (valid && lrank == 0) wc[warp * ndig + d] = __popc(peers);
    __syncthreads();
    if (valid) {
        int r = lrank;
        for (int w = 0; w < warp; ++w) r += wc[w * ndig + d];
        perm_out[O[(size_t)d * gridDim.x + blockIdx.x] + r] = src;
    }
}

__global__ void k_gather_events(const int32_t* __restrict__ perm, int64_t n,
                                const int32_t* __restrict__ a, const float* __restrict__ u,
                                const float* __restrict__ e, int32_t* __restrict__ a_s,
                                float* __restrict__ u_s, float* __restrict__ e_s,
                                int64_t* __restrict__ rank) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int32_t j = perm[r];
    a_s[r] = a[j];
    u_s[r] = u[j];
    e_s[r] = e[j];
    rank[j] = r;
}

lmosem_status counting_pass(lmosem_ctx* c, const Digit& dg, int ndig, const int32_t* perm_in,
                            int32_t* perm_out, int64_t n, int32_t* H, int32_t* tot) {
    int nblk = (int)((n + kSortThreads - 1) / kSortThreads);
    LMOSEM_PROF_BEGIN(c);
    k_hist<<<nblk, kSortThreads, ndig * sizeof(int32_t), c->stream>>>(dg, perm_in, n, ndig, H);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SORT);
    int64_t hn = (int64_t)ndig * nblk;
    int sblk = (int)((hn + kScanBlock * 4 - 1) / (kScanBlock * 4));
    LMOSEM_PROF_BEGIN(c);
    k_scan_local<<<sblk, kScanBlock, 0, c->stream>>>(H, hn, tot);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SORT);
    LMOSEM_PROF_BEGIN(c);
    k_scan_totals<<<1, kScanBlock, 0, c->stream>>>(tot, sblk);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SORT);
    LMOSEM_PROF_BEGIN(c);
    k_scan_add<<<(int)((hn + 255) / 256), 256, 0, c->stream>>>(H, hn, tot);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SORT);
    size_t smem = (size_t)(kSortThreads / 32) * ndig * sizeof(int32_t);
    LMOSEM_PROF_BEGIN(c);
    k_scatter<<<nblk, kSortThreads, smem, c->stream>>>(dg, perm_in, n, ndig, H, perm_out);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SORT);
    return LMOSEM_OK;
}

}  // namespace

lmosem_status validate_events(lmosem_ctx* c, const int32_t* d_angle, const float* d_u, const float* d_e,
                              int64_t n) {
    lmosem_status st;
    const float half = (float)(0.5 * c->n_bins * c->bin_mm);
    int32_t* d_bad = nullptr;
    Scratch tmp(c);
    if ((st = tmp.alloc(&d_bad, 1))) return st;
    LMOSEM_CK(c, cudaMemsetAsync(d_bad, 0, sizeof(int32_t), c->stream));
    LMOSEM_PROF_BEGIN(c);
    k_check_events<<<(int)((n + 255) / 256), 256, 0, c->stream>>>(
        d_angle, d_u, d_e, n, c->n_angles, half, (float)c->e_lo, (float)c->e_hi, d_bad);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SORT);
    int32_t bad = 0;
    LMOSEM_CK(c, cudaMemcpyAsync(&bad, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    if (bad) return fail(c, LMOSEM_EINVAL, std::to_string(bad) +
                                               " events have an angle, position or energy out of range");
    return LMOSEM_OK;
}

lmosem_status sort_events(lmosem_ctx* c, const int32_t* d_angle, const float* d_u,
                          const float* d_e, int64_t n, int n_subsets, const int64_t* h_offsets,
                          int n_real) {
    lmosem_status st;
    if ((st = validate_events(c, d_angle, d_u, d_e, n))) return st;
    const float half = (float)(0.5 * c->n_bins * c->bin_mm);

    const int group = (c->n_angles + n_subsets - 1) / n_subsets;
    const int ndig_a = n_subsets * group;
    // the stable scatter keeps one count per (warp, digit) in 48 KB of shared memory
    if (ndig_a > 1536 || n_real > 1536)
        return fail(c, LMOSEM_EINVAL, "too many angles or realisations for the event sort");
    int ndig = ndig_a > 2 * kUBins ? ndig_a : 2 * kUBins;
    ndig = ndig > n_real ? ndig : n_real;
    const int nblk = (int)((n + kSortThreads - 1) / kSortThreads);
    const int64_t hn = (int64_t)ndig * nblk;
    const int sblk = (int)((hn + kScanBlock * 4 - 1) / (kScanBlock * 4));
    int32_t *H = nullptr, *tot = nullptr, *p1 = nullptr, *p2 = nullptr, *cnt = nullptr;
    int64_t* d_off = nullptr;
    Scratch tmp(c);
    if ((st = tmp.alloc(&H, hn))) return st;
    if ((st = tmp.alloc(&tot, sblk))) return st;
    if ((st = tmp.alloc(&p1, n))) return st;
    if ((st = tmp.alloc(&cnt, (size_t)n_real * c->n_angles))) return st;
    if ((st = dev_alloc(c, &c->d_perm, n))) return st;
    if ((st = dev_alloc(c, &c->d_rank, n))) return st;
    if ((st = dev_alloc(c, &c->d_a_s, n))) return st;
    if ((st = dev_alloc(c, &c->d_u_s, n))) return st;
    if ((st = dev_alloc(c, &c->d_e_s, n))) return st;
    if (n_real > 1) {
        if ((st = tmp.alloc(&p2, n))) return st;
        if ((st = tmp.alloc(&d_off, n_real + 1))) return st;
        LMOSEM_CK(c, cudaMemcpyAsync(d_off, h_offsets, (n_real + 1) * sizeof(int64_t),
                                     cudaMemcpyHostToDevice, c->stream));
    }

    // stable passes, least significant key first: (energy class, position
    // bin), angle slot and, for several realisations, the realisation
    const float e_class = (float)(c->e0 * (1.0 - 0.5 * c->fwhm_frac));
    Digit d0{0, d_angle, d_u, half, n_subsets, group, d_off, n_real, d_e, e_class};
    Digit d1{1, d_angle, d_u, half, n_subsets, group, d_off, n_real, d_e, e_class};
    Digit d2{2, d_angle, d_u, half, n_subsets, group, d_off, n_real, d_e, e_class};
    if ((st = counting_pass(c, d0, 2 * kUBins, nullptr, p1, n, H, tot))) return st;
    if (n_real > 1) {
        if ((st = counting_pass(c, d1, ndig_a, p1, p2, n, H, tot))) return st;
        if ((st = counting_pass(c, d2, n_real, p2, c->d_perm, n, H, tot))) return st;
    } else {
        if ((st = counting_pass(c, d1, ndig_a, p1, c->d_perm, n, H, tot))) return st;
    }
    LMOSEM_PROF_BEGIN(c);
    k_gather_events<<<(int)((n + 255) / 256), 256, 0, c->stream>>>(
        c->d_perm, n, d_angle, d_u, d_e, c->d_a_s, c->d_u_s, c->d_e_s, c->d_rank);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SORT);
    LMOSEM_CK(c, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)n_real * c->n_angles, c->stream));
    LMOSEM_PROF_BEGIN(c);
    k_rs_hist<<<(int)((n + 255) / 256), 256, 0, c->stream>>>(c->d_a_s, n, d_off, n_real,
                                                             c->n_angles, cnt);
    LMOSEM_LAUNCHED(c, LMOSEM_K_SORT);

    std::vector<int32_t> h_cnt((size_t)n_real * c->n_angles);
    LMOSEM_CK(c, cudaMemcpyAsync(h_cnt.data(), cnt, h_cnt.size() * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));

    // rows of (realisation, angle) and of (realisation, subset), in sorted order
    c->n_real = n_real;
    c->h_real_row0.assign(n_real + 1, 0);
    c->h_angle_row0.assign((size_t)n_real * c->n_angles, 0);
    c->h_angle_cnt.assign((size_t)n_real * c->n_angles, 0);
    c->h_subset_row0.assign((size_t)n_real * (n_subsets + 1), 0);
    int64_t row = 0;
    for (int r = 0; r < n_real; ++r) {
        c->h_real_row0[r] = row;
        for (int s = 0; s < ndig_a; ++s) {
            if (s % group == 0) c->h_subset_row0[(size_t)r * (n_subsets + 1) + s / group] = row;
            int a = (s / group) + n_subsets * (s % group);
            if (a >= c->n_angles) continue;
            size_t k = (size_t)r * c->n_angles + a;
            c->h_angle_row0[k] = row;
            c->h_angle_cnt[k] = h_cnt[k];
            row += h_cnt[k];
        }
        c->h_subset_row0[(size_t)r * (n_subsets + 1) + n_subsets] = row;
    }
    c->h_real_row0[n_real] = row;
    if (row != n) return fail(c, LMOSEM_ECUDA, "event sort lost events");
    return LMOSEM_OK;
}

}  // namespace lmosem
