// C ABI of the lmosem library: argument validation, context ownership and
// the order of the hot-path steps.  Every numerical step runs in the
// kernels of the other translation units; this file only checks arguments,
// allocates, and enqueues.
#include <math.h>

#include <cmath>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "lmosem_internal.cuh"

namespace lmosem {

lmosem_status fail(lmosem_ctx* c, lmosem_status st, const std::string& msg) {
    if (c) c->err = msg;
    return st;
}

lmosem_status cuda_fail(lmosem_ctx* c, cudaError_t e, const char* what) {
    return fail(c, LMOSEM_ECUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                                     cudaGetErrorString(e) + ")");
}

static cudaEvent_t prof_event(lmosem_ctx* c) {
    if (!c->prof_pool.empty()) {
        cudaEvent_t e = c->prof_pool.back();
        c->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(lmosem_ctx* c) {
    if (c->capturing) return;
    c->prof_open = prof_event(c);
    cudaEventRecord(c->prof_open, c->stream);
}

void prof_end(lmosem_ctx* c, int cls) {
    if (!c->prof_open) return;
    cudaEvent_t b = prof_event(c);
    cudaEventRecord(b, c->stream);
    c->prof.push_back({cls, c->prof_open, b});
    c->prof_open = nullptr;
}

namespace {

__global__ void k_count_nonfinite(const float* __restrict__ f, int n, int* __restrict__ bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !isfinite(f[i])) atomicAdd(bad, 1);
}

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

void drop_graph(lmosem_ctx* c) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
    c->graph_f = nullptr;
    if (c->bgraph_exec) cudaGraphExecDestroy(c->bgraph_exec);
    c->bgraph_exec = nullptr;
    c->bgraph_f = nullptr;
}

void free_model(lmosem_ctx* c) {
    drop_graph(c);
    dev_free(c, &c->d_model);
    dev_free(c, &c->d_scale);
    dev_free(c, &c->d_stage);
    dev_free(c, &c->d_perm);
    dev_free(c, &c->d_rank);
    dev_free(c, &c->d_u_s);
    dev_free(c, &c->d_e_s);
    dev_free(c, &c->d_a_s);
    dev_free(c, &c->d_angle_row0);
    dev_free(c, &c->d_angle_cnt);
    dev_free(c, &c->d_tile_prefix);
    dev_free(c, &c->d_wtab);
    dev_free(c, &c->d_bsub_row0);
    dev_free(c, &c->d_breal_row0);
    dev_free(c, &c->d_bclaim);
    dev_free(c, &c->d_bdone);
    dev_free(c, &c->d_bpart_batch);
    dev_free(c, &c->d_weight);
    c->n_counts = 0.0;
    c->bpart_batch_floats = 0;
    c->batch_model = false;
    c->use_surrogate = false;
    c->sur_checked = false;
    c->sur_exact = false;
    c->n_real = 1;
    c->fmt = -1;
    c->J = 0;
    c->n_subsets = 0;
}

lmosem_status check_events_args(lmosem_ctx* c, const int32_t* d_angle, const float* d_u,
                                const float* d_e, int64_t n_events, int32_t n_subsets,
                                lmosem_model_fmt fmt) {
    if (!d_angle || !d_u || !d_e) return fail(c, LMOSEM_EINVAL, "null event array");
    if (n_events < 1 || n_events >= (int64_t(1) << 31))
        return fail(c, LMOSEM_EINVAL, "n_events must be in [1, 2^31)");
    if (n_subsets < 1 || n_subsets > c->n_angles)
        return fail(c, LMOSEM_EINVAL, "n_subsets must be in [1, n_angles]");
    if (fmt != LMOSEM_MODEL_FP32 && fmt != LMOSEM_MODEL_FP16_SCALED && fmt != LMOSEM_MODEL_BF16_SCALED &&
        fmt != LMOSEM_MODEL_SURROGATE_FP32)
        return fail(c, LMOSEM_EINVAL, "unknown model format");
    if (fmt == LMOSEM_MODEL_SURROGATE_FP32 && !c->d_surrogate)
        return fail(c, LMOSEM_ESTATE, "no surrogate loaded (lmosem_surrogate_load)");
    return LMOSEM_OK;
}

// The energy gate's cut from the judge's sampled rows (squared difference
// and squared exact norm per row, and the rows' event energies): the top of
// the highest bin whose mean per-row relative L2 error exceeds the gate's
// tolerance (a NaN mean fails), infinity when that is the window's last bin,
// the window's lower edge when no bin fails.
double gate_cut(const lmosem_ctx* c, const std::vector<double>& sums, const std::vector<float>& ev) {
    const int nb = std::max(1, (int)ceil((c->e_hi - c->e_lo) / c->sur_gate_bin - 1e-9));
    std::vector<double> esum(nb, 0.0);
    std::vector<int> cnt(nb, 0);
    for (size_t k = 0; k < ev.size(); ++k) {
        const double d2 = sums[2 * k], e2 = sums[2 * k + 1];
        const double r = e2 > 0.0 ? sqrt(d2 / e2) : (d2 > 0.0 ? INFINITY : 0.0);
        const int b = std::min(nb - 1, std::max(0, (int)floor(((double)ev[k] - c->e_lo) / c->sur_gate_bin)));
        esum[b] += r;
        ++cnt[b];
    }
    int top = -1;
    for (int b = 0; b < nb; ++b)
        if (cnt[b] > 0 && !(esum[b] / cnt[b] <= c->sur_gate_tol)) top = b;
    if (top < 0) return c->e_lo;
    return top + 1 >= nb ? INFINITY : c->e_lo + (top + 1) * c->sur_gate_bin;
}

// The surrogate-form model and its exact check.  The judge compares the
// network's rows with the exact path sum's on a sample of rows.  Without the
// energy gate every row is built by the network first.  With it the sample's
// rows are built first; the judge's cut then decides which rows the network
// builds (event energy at or above the cut) and which the exact path sum
// builds (below), and the check's error is taken with the latter exact.
// Above the check's tolerance the whole model is rebuilt exactly.
lmosem_status build_checked_surrogate(lmosem_ctx* c) {
    const bool gate = c->sur_tol > 0.0 && c->sur_gate_tol > 0.0;
    lmosem_status st;
    if (!gate) {
        if ((st = build_model_rows(c))) return st;
    } else {
        const std::vector<int64_t> rows = judge_sample_rows(c);
        int64_t* d_rows = nullptr;
        Scratch tmp(c);
        if ((st = tmp.alloc(&d_rows, rows.size()))) return st;
        LMOSEM_CK(c, cudaMemcpyAsync(d_rows, rows.data(), rows.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                                     c->stream));
        if ((st = build_model_surrogate_rows(c, d_rows, (int64_t)rows.size()))) return st;
    }
    double err = 0.0, mx = 0.0;
    std::vector<double> sums;
    std::vector<float> ev;
    if ((st = judge_surrogate(c, &err, &mx, &sums, &ev))) return st;
    c->sur_checked = true;
    c->sur_exact = false;
    c->sur_cut = c->e_lo;
    c->sur_frac_exact = 0.0;
    if (gate) {
        const double cut = gate_cut(c, sums, ev);
        int64_t n_net = 0, n_exact = 0;
        if ((st = build_surrogate_rows_above(c, cut, &n_net))) return st;
        if ((st = rebuild_rows_below(c, cut, &n_exact))) return st;
        c->sur_cut = std::min(cut, c->e_hi);
        c->sur_frac_exact = (double)n_exact / (double)c->J;
        c->sur_exact = n_exact == c->J;
        double d2 = 0.0, e2 = 0.0;
        mx = 0.0;
        for (size_t k = 0; k < ev.size(); ++k) {
            e2 += sums[2 * k + 1];
            if ((double)ev[k] < cut) continue;  // an exact row
            d2 += sums[2 * k];
            if (sums[2 * k + 1] > 0.0) mx = std::max(mx, sqrt(sums[2 * k] / sums[2 * k + 1]));
            else if (sums[2 * k] > 0.0) mx = INFINITY;
        }
        err = e2 > 0.0 ? sqrt(d2 / e2) : (d2 > 0.0 ? INFINITY : 0.0);
    }
    c->sur_err = err;
    c->sur_row_max = mx;
    if (c->sur_tol > 0.0 && !(err <= c->sur_tol)) {  // a NaN error rebuilds too
        c->use_surrogate = false;
        if ((st = build_model_rows(c))) return st;
        c->sur_exact = true;
        c->sur_cut = c->e_hi;
        c->sur_frac_exact = 1.0;
    }
    return LMOSEM_OK;
}

// allocation, sort and row build shared by the single and the batched model
lmosem_status build_model_common(lmosem_ctx* c, const int32_t* d_angle, const float* d_u_mm,
                                 const float* d_e_kev, int64_t n_events, int32_t n_subsets,
                                 lmosem_model_fmt fmt, const int64_t* h_offsets, int n_real) {
    free_model(c);
    // the surrogate form is stored as FP32 rows; only their scatter part differs
    const bool sur = fmt == LMOSEM_MODEL_SURROGATE_FP32;
    if (sur) fmt = LMOSEM_MODEL_FP32;
    c->fmt = fmt;
    c->use_surrogate = sur;
    c->J = n_events;
    c->n_subsets = n_subsets;
    c->ld_model = (c->n_sup + 31) / 32 * 32;
    lmosem_status st;
    size_t elem = fmt == LMOSEM_MODEL_FP32 ? 4 : 2;
    {
        void* p = nullptr;
        cudaError_t e = cudaMallocAsync(&p, (size_t)n_events * c->ld_model * elem, c->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_model(c);
            return fail(c, LMOSEM_ENOMEM, "model of " +
                                              std::to_string((size_t)n_events * c->ld_model * elem) +
                                              " bytes does not fit: " + cudaGetErrorString(e));
        }
        c->d_model = p;
    }
    if (fmt != LMOSEM_MODEL_FP32 && (st = dev_alloc(c, &c->d_scale, n_events))) {
        free_model(c);
        return st;
    }
    if ((st = sort_events(c, d_angle, d_u_mm, d_e_kev, n_events, n_subsets, h_offsets, n_real))) {
        free_model(c);
        return st;
    }
    if ((st = sur ? build_checked_surrogate(c) : build_model_rows(c))) {
        free_model(c);
        return st;
    }
    if (!c->d_bpart && (st = setup_pass(c))) return st;
    return LMOSEM_OK;
}

}  // namespace
}  // namespace lmosem

using namespace lmosem;

extern "C" {

const char* lmosem_status_string(lmosem_status st) {
    switch (st) {
        case LMOSEM_OK: return "ok";
        case LMOSEM_EINVAL: return "invalid argument";
        case LMOSEM_ENOMEM: return "out of device memory";
        case LMOSEM_ECUDA: return "CUDA error";
        case LMOSEM_ETIMEOUT: return "device wait timed out";
        case LMOSEM_ENUMERIC: return "non-finite value";
        case LMOSEM_ESTATE: return "called out of order";
        case LMOSEM_ENOTIMPL: return "not implemented";
    }
    return "unknown status";
}

const char* lmosem_last_error(const lmosem_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int32_t lmosem_n_support(const lmosem_ctx* ctx) { return ctx ? ctx->n_sup : 0; }
int32_t lmosem_n_scatter(const lmosem_ctx* ctx) { return ctx ? ctx->n_scat : 0; }
int64_t lmosem_launch_count(const lmosem_ctx* ctx) { return ctx ? ctx->launches : 0; }

lmosem_status lmosem_set_wait_budget(lmosem_ctx* c, int64_t cycles) {
    if (!c) return LMOSEM_EINVAL;
    if (cycles < 0) return fail(c, LMOSEM_EINVAL, "negative wait budget");
    c->wait_budget = cycles > 0 ? cycles : 2000000000LL;
    return LMOSEM_OK;
}

lmosem_status lmosem_model_terms(lmosem_ctx* c, int64_t* h_terms) {
    if (!c || !h_terms) return LMOSEM_EINVAL;
    if (!c->terms_valid || !c->d_terms) return fail(c, LMOSEM_EINVAL, "no exact model build to count");
    unsigned long long v = 0;
    LMOSEM_CK(c, cudaMemcpyAsync(&v, c->d_terms, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    *h_terms = (int64_t)v;
    return LMOSEM_OK;
}

int64_t lmosem_model_bytes(const lmosem_ctx* ctx) {
    if (!ctx || ctx->fmt < 0) return 0;
    int64_t elem = ctx->fmt == LMOSEM_MODEL_FP32 ? 4 : 2;
    return ctx->J * ctx->ld_model * elem + (ctx->fmt == LMOSEM_MODEL_FP32 ? 0 : ctx->J * 4);
}

lmosem_status lmosem_support(const lmosem_ctx* ctx, int32_t* h_out) {
    if (!ctx || !h_out) return LMOSEM_EINVAL;
    std::copy(ctx->h_sup.begin(), ctx->h_sup.end(), h_out);
    return LMOSEM_OK;
}

void lmosem_destroy(lmosem_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_model(c);
    dev_free(c, &c->d_wtab_all);
    dev_free(c, &c->d_mu);
    dev_free(c, &c->d_sup);
    dev_free(c, &c->d_scat);
    dev_free(c, &c->d_scat_geo);
    dev_free(c, &c->d_trig);
    dev_free(c, &c->d_l_edge);
    dev_free(c, &c->d_line);
    dev_free(c, &c->d_l_pair);
    dev_free(c, &c->d_compton);
    dev_free(c, &c->d_mpar);
    dev_free(c, &c->d_ppar);
    dev_free(c, &c->d_du_m);
    dev_free(c, &c->d_sens);
    dev_free(c, &c->d_sens_angle);
    dev_free(c, &c->d_bpart);
    dev_free(c, &c->d_coop);
    c->coop_words = 0;
    dev_free(c, &c->d_llpart);
    dev_free(c, &c->d_scalar);
    dev_free(c, &c->d_terms);
    dev_free(c, &c->d_status);
    dev_free(c, &c->d_surrogate);
    for (auto& r : c->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->prof_pool) cudaEventDestroy(e);
    if (c->prof_open) cudaEventDestroy(c->prof_open);
    delete c;
}

lmosem_status lmosem_create(const lmosem_object* obj, const lmosem_geometry* geom,
                            const lmosem_energy* en, const lmosem_options* opts, void* stream,
                            lmosem_ctx** out) {
    if (!out) return LMOSEM_EINVAL;
    *out = nullptr;
    if (!obj || !geom || !en || !obj->h_mu_per_mm) return LMOSEM_EINVAL;
    if (obj->nx < 1 || obj->ny < 1 || obj->nx > 2048 || obj->ny > 2048 || !finite_pos(obj->pixel_mm))
        return LMOSEM_EINVAL;
    if (geom->n_angles < 1 || geom->n_angles > 1536 || geom->n_bins < 1 || !finite_pos(geom->bin_mm) ||
        !finite_pos(geom->radius_mm) || !finite_pos(geom->coll_fwhm0_mm) ||
        !isfinite(geom->coll_fwhm_slope) || geom->coll_fwhm_slope < 0 || !isfinite(geom->angle0_rad))
        return LMOSEM_EINVAL;
    if (!finite_pos(en->e0_kev) || !finite_pos(en->fwhm_frac_e0) || !finite_pos(en->e_lo_kev) ||
        !isfinite(en->e_hi_kev) || en->e_hi_kev <= en->e_lo_kev)
        return LMOSEM_EINVAL;
    float ks = opts && opts->k_sigma != 0.0f ? opts->k_sigma : 6.0f;
    if (!(ks > 0.0f && ks <= 20.0f)) return LMOSEM_EINVAL;
    float es = opts && opts->e_sigma != 0.0f ? opts->e_sigma : 6.0f;
    if (!(es <= 20.0f)) return LMOSEM_EINVAL;  // also rejects NaN

    lmosem_ctx* c = new (std::nothrow) lmosem_ctx();
    if (!c) return LMOSEM_ENOMEM;
    c->stream = (cudaStream_t)stream;
    {  // keep up to kPoolKeepBytes of freed device memory cached in the default pool
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = kPoolKeepBytes;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    }
    c->nx = obj->nx;
    c->ny = obj->ny;
    c->npix = obj->nx * obj->ny;
    c->dpx = obj->pixel_mm;
    c->n_angles = geom->n_angles;
    c->angle0 = geom->angle0_rad;
    c->n_bins = geom->n_bins;
    c->bin_mm = geom->bin_mm;
    c->radius = geom->radius_mm;
    c->fwhm0 = geom->coll_fwhm0_mm;
    c->fwhm_slope = geom->coll_fwhm_slope;
    c->e0 = en->e0_kev;
    c->fwhm_frac = en->fwhm_frac_e0;
    c->e_lo = en->e_lo_kev;
    c->e_hi = en->e_hi_kev;
    c->k_sigma = ks;
    c->e_sigma = es > 0.0f ? es : 0.0f;
    if (opts && opts->table_budget_bytes > 0) c->table_budget = opts->table_budget_bytes;
    c->profile = opts ? opts->profile : 0;
    if (c->profile < 0 || c->profile > 2) {
        delete c;
        return LMOSEM_EINVAL;
    }
    if (opts && opts->wait_budget_cycles > 0) c->wait_budget = opts->wait_budget_cycles;
    if (opts) {
        if (opts->pass_variant < 0 || opts->pass_variant > 4 || opts->ring_rows < 0 ||
            opts->ring_stages < 0) {
            delete c;
            return LMOSEM_EINVAL;
        }
        c->pass_variant = opts->pass_variant;
        c->ring_rows = opts->ring_rows;
        c->ring_stages = opts->ring_stages;
        if (opts->surrogate_kernel < 0 || opts->surrogate_kernel > 2) {
            delete c;
            return LMOSEM_EINVAL;
        }
        c->surrogate_kernel = opts->surrogate_kernel;
        if (opts->prefetch_groups < -1 || opts->prefetch_groups > 16) {
            delete c;
            return LMOSEM_EINVAL;
        }
        c->prefetch_groups = opts->prefetch_groups;
    }

    std::vector<float> mu(c->npix);
    double rmax = 0.0;
    for (int p = 0; p < c->npix; ++p) {
        double v = obj->h_mu_per_mm[p];
        if (!isfinite(v) || v < 0.0) {
            delete c;
            return LMOSEM_EINVAL;
        }
        mu[p] = (float)v;
        bool sup = obj->h_support ? obj->h_support[p] != 0 : v > 0.0;
        if (sup) c->h_sup.push_back(p);
        if (v > 0.0) c->h_scat.push_back(p);
        if (sup || v > 0.0) {
            double x = (p % c->nx + 0.5 - 0.5 * c->nx) * c->dpx;
            double y = (p / c->nx + 0.5 - 0.5 * c->ny) * c->dpx;
            rmax = std::max(rmax, sqrt(x * x + y * y));
        }
    }
    c->n_sup = (int)c->h_sup.size();
    c->n_scat = (int)c->h_scat.size();
    if (c->n_sup == 0) {
        lmosem_status st = fail(c, LMOSEM_EINVAL, "empty emission support");
        delete c;
        return st;
    }
    if (c->n_scat > 32768) {
        delete c;
        return LMOSEM_EINVAL;
    }
    if (geom->radius_mm <= rmax) {
        delete c;
        return LMOSEM_EINVAL;
    }
    c->ld_w = (c->n_sup + kTN - 1) / kTN * kTN;

    lmosem_status st;
    if ((st = dev_alloc(c, &c->d_mu, c->npix)) || (st = dev_alloc(c, &c->d_sup, c->n_sup)) ||
        (st = dev_alloc(c, &c->d_scat, std::max(1, c->n_scat))) ||
        (st = dev_alloc(c, &c->d_scat_geo, std::max(1, c->n_scat)))) {
        lmosem_destroy(c);
        return st;
    }
    cudaError_t e = cudaMemcpyAsync(c->d_mu, mu.data(), mu.size() * sizeof(float),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_sup, c->h_sup.data(), c->n_sup * sizeof(int32_t),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && c->n_scat)
        e = cudaMemcpyAsync(c->d_scat, c->h_scat.data(), c->n_scat * sizeof(int32_t),
                            cudaMemcpyHostToDevice, c->stream);
    // scatter-pixel centres: (ix + 1/2 - nx/2) is exact in FP32, so the one
    // rounding of the product by the pixel size gives the device's bits
    std::vector<float4> geo(c->n_scat);
    for (int k = 0; k < c->n_scat; ++k) {
        const int pm = c->h_scat[k];
        const float fx = (float)(pm % c->nx) + 0.5f - 0.5f * (float)c->nx;
        const float fy = (float)(pm / c->nx) + 0.5f - 0.5f * (float)c->ny;
        int32_t bits = pm;
        float fbits;
        memcpy(&fbits, &bits, sizeof(float));
        geo[k] = make_float4(fx * (float)c->dpx, fy * (float)c->dpx, mu[pm], fbits);
    }
    if (e == cudaSuccess && c->n_scat)
        e = cudaMemcpyAsync(c->d_scat_geo, geo.data(), c->n_scat * sizeof(float4),
                            cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) {
        cuda_fail(c, e, "copy of the mu-map");
        lmosem_destroy(c);
        return LMOSEM_ECUDA;
    }
    if ((st = build_tables(c))) {
        fprintf(stderr, "lmosem_create: %s\n", c->err.c_str());
        lmosem_destroy(c);
        return st;
    }
    *out = c;
    return LMOSEM_OK;
}

lmosem_status lmosem_sensitivity(lmosem_ctx* c, int32_t n_subsets, double* d_sens) {
    if (!c) return LMOSEM_EINVAL;
    if (n_subsets < 1 || n_subsets > c->n_angles)
        return fail(c, LMOSEM_EINVAL, "n_subsets must be in [1, n_angles]");
    drop_graph(c);  // the captured iteration reads the sensitivity buffer
    lmosem_status st = compute_sensitivity(c, n_subsets);
    if (st) return st;
    if (d_sens)
        LMOSEM_CK(c, cudaMemcpyAsync(d_sens, c->d_sens, sizeof(double) * (size_t)n_subsets * c->n_sup,
                                     cudaMemcpyDeviceToDevice, c->stream));
    return LMOSEM_OK;
}

lmosem_status lmosem_build_model(lmosem_ctx* c, const int32_t* d_angle, const float* d_u_mm,
                                 const float* d_e_kev, int64_t n_events, int32_t n_subsets,
                                 lmosem_model_fmt fmt) {
    if (!c) return LMOSEM_EINVAL;
    lmosem_status st = check_events_args(c, d_angle, d_u_mm, d_e_kev, n_events, n_subsets, fmt);
    if (st) return st;
    return build_model_common(c, d_angle, d_u_mm, d_e_kev, n_events, n_subsets, fmt, nullptr, 1);
}

lmosem_status lmosem_build_model_binned(lmosem_ctx* c, const float* d_counts, int32_t n_ebins,
                                        const double* h_e_edges, int32_t n_subsets, lmosem_model_fmt fmt) {
    if (!c) return LMOSEM_EINVAL;
    if (!d_counts || !h_e_edges) return fail(c, LMOSEM_EINVAL, "null counts or energy edges");
    if (n_ebins < 1 || n_ebins > 8) return fail(c, LMOSEM_EINVAL, "n_ebins must be in 1..8");
    if (n_subsets < 1 || n_subsets > c->n_angles)
        return fail(c, LMOSEM_EINVAL, "n_subsets must be in [1, n_angles]");
    if (fmt != LMOSEM_MODEL_FP32) return fail(c, LMOSEM_ENOTIMPL, "the binned model is cached as FP32 only");
    for (int k = 0; k <= n_ebins; ++k)
        if (!std::isfinite(h_e_edges[k]) || (k > 0 && !(h_e_edges[k] > h_e_edges[k - 1])))
            return fail(c, LMOSEM_EINVAL, "energy edges must be finite and increasing");
    const double tol = 1e-9 * c->e_hi;
    if (fabs(h_e_edges[0] - c->e_lo) > tol || fabs(h_e_edges[n_ebins] - c->e_hi) > tol)
        return fail(c, LMOSEM_EINVAL, "energy edges must span the window [e_lo, e_hi]");

    // counts to the host, checked, and the positive bins in sorted-row order:
    // subsets in index order, their angles increasing, then (position, energy) bin
    const int K = n_ebins, NB = c->n_bins, NA = c->n_angles;
    const size_t nbins = (size_t)NA * NB * K;
    std::vector<float> h(nbins);
    LMOSEM_CK(c, cudaMemcpyAsync(h.data(), d_counts, nbins * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    int64_t n_rows = 0;
    double total = 0.0;
    for (size_t i = 0; i < nbins; ++i) {
        if (!std::isfinite(h[i]) || h[i] < 0.0f) return fail(c, LMOSEM_EINVAL, "counts must be finite and >= 0");
        if (h[i] > 0.0f) {
            ++n_rows;
            total += h[i];
        }
    }
    if (n_rows == 0) return fail(c, LMOSEM_EINVAL, "no positive count");
    std::vector<int32_t> rowmap(nbins, -1);
    std::vector<float> weight(n_rows);
    std::vector<int64_t> angle_row0(NA, 0), angle_cnt(NA, 0), subset_row0(n_subsets + 1, 0);
    int64_t r = 0;
    for (int i = 0; i < n_subsets; ++i) {
        subset_row0[i] = r;
        for (int a = i; a < NA; a += n_subsets) {
            angle_row0[a] = r;
            for (size_t q = (size_t)a * NB * K; q < (size_t)(a + 1) * NB * K; ++q)
                if (h[q] > 0.0f) {
                    rowmap[q] = (int32_t)r;
                    weight[r++] = h[q];
                }
            angle_cnt[a] = r - angle_row0[a];
        }
    }
    subset_row0[n_subsets] = r;
    std::vector<int64_t> rank;  // ordinal of a positive bin in dense order -> row
    rank.reserve(n_rows);
    for (size_t q = 0; q < nbins; ++q)
        if (rowmap[q] >= 0) rank.push_back(rowmap[q]);

    free_model(c);
    c->fmt = LMOSEM_MODEL_FP32;
    c->use_surrogate = false;
    c->J = n_rows;
    c->n_subsets = n_subsets;
    c->ld_model = (c->n_sup + 31) / 32 * 32;
    c->n_real = 1;
    c->h_real_row0 = {0, n_rows};
    c->h_angle_row0 = angle_row0;
    c->h_angle_cnt = angle_cnt;
    c->h_subset_row0 = subset_row0;
    lmosem_status st;
    {
        void* p = nullptr;
        cudaError_t e = cudaMallocAsync(&p, (size_t)n_rows * c->ld_model * sizeof(float), c->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_model(c);
            return fail(c, LMOSEM_ENOMEM, "binned model does not fit");
        }
        c->d_model = p;
    }
    Scratch tmp(c);
    int32_t* d_rowmap = nullptr;
    if ((st = dev_alloc(c, &c->d_weight, (size_t)n_rows)) || (st = dev_alloc(c, &c->d_rank, (size_t)n_rows)) ||
        (st = tmp.alloc(&d_rowmap, nbins))) {
        free_model(c);
        return st;
    }
    LMOSEM_CK(c, cudaMemcpyAsync(c->d_weight, weight.data(), n_rows * sizeof(float), cudaMemcpyHostToDevice,
                                 c->stream));
    LMOSEM_CK(c, cudaMemcpyAsync(c->d_rank, rank.data(), n_rows * sizeof(int64_t), cudaMemcpyHostToDevice,
                                 c->stream));
    LMOSEM_CK(c, cudaMemcpyAsync(d_rowmap, rowmap.data(), nbins * sizeof(int32_t), cudaMemcpyHostToDevice,
                                 c->stream));
    if ((st = build_binned_rows(c, d_rowmap, K, h_e_edges))) {
        free_model(c);
        return st;
    }
    c->n_counts = total;
    if (!c->d_bpart && (st = setup_pass(c))) return st;
    return LMOSEM_OK;
}

lmosem_status lmosem_build_model_batch(lmosem_ctx* c, const int32_t* d_angle, const float* d_u_mm,
                                       const float* d_e_kev, const int64_t* h_event_offsets,
                                       int32_t n_real, int32_t n_subsets, lmosem_model_fmt fmt) {
    if (!c) return LMOSEM_EINVAL;
    if (!h_event_offsets || n_real < 1 || n_real > 1536)
        return fail(c, LMOSEM_EINVAL, "need 1..1536 realisations and their event offsets");
    const int64_t n_events = h_event_offsets[n_real];
    if (h_event_offsets[0] != 0) return fail(c, LMOSEM_EINVAL, "event offsets must start at 0");
    for (int r = 0; r < n_real; ++r)
        if (h_event_offsets[r + 1] < h_event_offsets[r])
            return fail(c, LMOSEM_EINVAL, "event offsets must not decrease");
    lmosem_status st = check_events_args(c, d_angle, d_u_mm, d_e_kev, n_events, n_subsets, fmt);
    if (st) return st;
    if (fmt != LMOSEM_MODEL_FP32)
        return fail(c, LMOSEM_ENOTIMPL, "the batched model is cached as FP32 only");
    if ((st = build_model_common(c, d_angle, d_u_mm, d_e_kev, n_events, n_subsets, fmt,
                                 h_event_offsets, n_real)))
        return st;
    if ((st = setup_batch(c))) {
        free_model(c);
        return st;
    }
    c->batch_model = true;
    return LMOSEM_OK;
}

lmosem_status lmosem_init_image_batch(lmosem_ctx* c, double T, float* d_f) {
    if (!c) return LMOSEM_EINVAL;
    if (!d_f || !finite_pos(T)) return fail(c, LMOSEM_EINVAL, "bad image pointer or acquisition time");
    if (!c->batch_model || c->sens_subsets != c->n_subsets)
        return fail(c, LMOSEM_ESTATE, "needs a batched model and a matching sensitivity");
    return run_init_batch(c, T, d_f);
}

lmosem_status lmosem_iterate_batch(lmosem_ctx* c, int32_t n_iters, double T, float* d_f) {
    if (!c) return LMOSEM_EINVAL;
    if (!d_f || n_iters < 0 || !finite_pos(T))
        return fail(c, LMOSEM_EINVAL, "bad image pointer, iteration count or acquisition time");
    if (!c->batch_model || c->sens_subsets != c->n_subsets)
        return fail(c, LMOSEM_ESTATE, "needs a batched model and a matching sensitivity");
    if (n_iters == 0) return LMOSEM_OK;
    LMOSEM_CK(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    lmosem_status st = run_batch(c, n_iters, T, d_f);
    if (st) return st;
    int h = 0;
    LMOSEM_CK(c, cudaMemcpyAsync(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    if (h) return fail(c, LMOSEM_ETIMEOUT, "a bounded device wait of the batched pass ran out");
    return LMOSEM_OK;
}

lmosem_status lmosem_autotune_batch(lmosem_ctx* c, double T, const float* d_f, int32_t* h_choice) {
    if (!c) return LMOSEM_EINVAL;
    if (!d_f || !finite_pos(T)) return fail(c, LMOSEM_EINVAL, "bad image pointer or acquisition time");
    if (!c->batch_model || c->sens_subsets != c->n_subsets)
        return fail(c, LMOSEM_ESTATE, "needs a batched model and a matching sensitivity");
    return run_autotune_batch(c, T, d_f, h_choice);
}

lmosem_status lmosem_set_batch_tiles(lmosem_ctx* c, int32_t chunk_rows, int32_t ctas_per_sm) {
    if (!c) return LMOSEM_EINVAL;
    if (chunk_rows < 8 || chunk_rows > (1 << 20) || ctas_per_sm < 1 || ctas_per_sm > 16)
        return fail(c, LMOSEM_EINVAL, "chunk_rows in [8, 2^20], ctas_per_sm in [1, 16]");
    c->batch_chunk_rows = chunk_rows;
    c->batch_ctas_per_sm = ctas_per_sm;
    return LMOSEM_OK;
}

lmosem_status lmosem_init_image(lmosem_ctx* c, double T, float* d_f) {
    if (!c) return LMOSEM_EINVAL;
    if (!d_f || !finite_pos(T)) return fail(c, LMOSEM_EINVAL, "bad image pointer or acquisition time");
    if (c->fmt < 0 || !c->sens_subsets) return fail(c, LMOSEM_ESTATE, "needs a model and a sensitivity");
    if (c->batch_model) return fail(c, LMOSEM_ESTATE, "a batched model takes lmosem_init_image_batch");
    return run_init_image(c, T, d_f);
}

lmosem_status lmosem_iterate(lmosem_ctx* c, int32_t n_iters, double T, float* d_f, double* d_ll) {
    if (!c) return LMOSEM_EINVAL;
    if (!d_f || n_iters < 0 || !finite_pos(T))
        return fail(c, LMOSEM_EINVAL, "bad image pointer, iteration count or acquisition time");
    if (c->fmt < 0) return fail(c, LMOSEM_ESTATE, "no model built");
    if (c->batch_model) return fail(c, LMOSEM_ESTATE, "a batched model takes lmosem_iterate_batch");
    if (c->sens_subsets != c->n_subsets)
        return fail(c, LMOSEM_ESTATE, "sensitivity missing or for another subset count");
    LMOSEM_CK(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    lmosem_status st = run_iterations(c, n_iters, T, d_f, d_ll);
    if (st) return st;
    // status word and non-finite count: [0] wait timeouts, [1] non-finite pixels
    int* bad = c->d_status + 1;
    LMOSEM_CK(c, cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
    LMOSEM_PROF_BEGIN(c);
    k_count_nonfinite<<<(c->n_sup + 255) / 256, 256, 0, c->stream>>>(d_f, c->n_sup, bad);
    LMOSEM_LAUNCHED(c, LMOSEM_K_OTHER);
    int h[2] = {0, 0};
    LMOSEM_CK(c, cudaMemcpyAsync(h, c->d_status, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    if (h[0])
        return fail(c, LMOSEM_ETIMEOUT,
                    "a bounded device wait ran out; the image may hold the sub-iterations finished before it");
    if (h[1]) return fail(c, LMOSEM_ENUMERIC, std::to_string(h[1]) + " non-finite image values");
    return LMOSEM_OK;
}

lmosem_status lmosem_subset_totals(lmosem_ctx* c, double T, const float* d_f, double* d_out) {
    if (!c) return LMOSEM_EINVAL;
    if (!d_f || !d_out || !finite_pos(T)) return fail(c, LMOSEM_EINVAL, "bad arguments");
    if (c->sens_subsets < 1 || (c->fmt >= 0 && c->sens_subsets != c->n_subsets))
        return fail(c, LMOSEM_ESTATE, "needs a sensitivity for the model's subset count");
    return run_subset_totals(c, T, d_f, d_out);
}

lmosem_status lmosem_loglik(lmosem_ctx* c, double T, const float* d_f, double* d_out) {
    if (!c) return LMOSEM_EINVAL;
    if (!d_f || !d_out || !finite_pos(T)) return fail(c, LMOSEM_EINVAL, "bad arguments");
    if (c->fmt < 0 || c->sens_subsets != c->n_subsets)
        return fail(c, LMOSEM_ESTATE, "needs a model and a matching sensitivity");
    if (c->batch_model) return fail(c, LMOSEM_ESTATE, "the log-likelihood takes a single-data-set model");
    LMOSEM_CK(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    lmosem_status st = run_loglik(c, T, d_f, d_out);
    if (st) return st;
    int h = 0;
    LMOSEM_CK(c, cudaMemcpyAsync(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    if (h) return fail(c, LMOSEM_ETIMEOUT, "a bounded device wait ran out");
    return LMOSEM_OK;
}

lmosem_status lmosem_reconstruct(lmosem_ctx* c, const int32_t* h_angle, const float* h_u_mm,
                                 const float* h_e_kev, int64_t n_events, int32_t n_subsets,
                                 lmosem_model_fmt fmt, int32_t n_iters, double T, float* h_f,
                                 double* h_loglik) {
    if (!c) return LMOSEM_EINVAL;
    if (!h_angle || !h_u_mm || !h_e_kev || !h_f) return fail(c, LMOSEM_EINVAL, "null host buffer");
    if (n_events < 1 || n_events >= (int64_t(1) << 31))
        return fail(c, LMOSEM_EINVAL, "n_events must be in [1, 2^31)");
    if (n_iters < 0 || !finite_pos(T))
        return fail(c, LMOSEM_EINVAL, "bad iteration count or acquisition time");
    int32_t* d_a = nullptr;
    float* d_u = nullptr;
    float* d_e = nullptr;
    float* d_f = nullptr;
    double* d_ll = nullptr;
    Scratch tmp(c);
    lmosem_status st;
    if ((st = tmp.alloc(&d_a, (size_t)n_events)) || (st = tmp.alloc(&d_u, (size_t)n_events)) ||
        (st = tmp.alloc(&d_e, (size_t)n_events)) || (st = tmp.alloc(&d_f, (size_t)c->n_sup)) ||
        (st = tmp.alloc(&d_ll, 1)))
        return st;
    const size_t n = (size_t)n_events;
    LMOSEM_CK(c, cudaMemcpyAsync(d_a, h_angle, n * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    LMOSEM_CK(c, cudaMemcpyAsync(d_u, h_u_mm, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    LMOSEM_CK(c, cudaMemcpyAsync(d_e, h_e_kev, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    if ((st = lmosem_sensitivity(c, n_subsets, nullptr)) ||
        (st = lmosem_build_model(c, d_a, d_u, d_e, n_events, n_subsets, fmt)) ||
        (st = lmosem_init_image(c, T, d_f)) || (st = lmosem_iterate(c, n_iters, T, d_f, nullptr)) ||
        (h_loglik && (st = lmosem_loglik(c, T, d_f, d_ll)))) {
        drop_graph(c);
        return st;
    }
    // the captured iteration graph refers to d_f, which is released on return
    drop_graph(c);
    LMOSEM_CK(c, cudaMemcpyAsync(h_f, d_f, sizeof(float) * (size_t)c->n_sup, cudaMemcpyDeviceToHost,
                                 c->stream));
    if (h_loglik)
        LMOSEM_CK(c, cudaMemcpyAsync(h_loglik, d_ll, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    return LMOSEM_OK;
}

lmosem_status lmosem_profile_read(lmosem_ctx* c, double* h_ms, int64_t* h_launches) {
    if (!c || !h_ms || !h_launches) return LMOSEM_EINVAL;
    if (!c->profile) return fail(c, LMOSEM_ESTATE, "profiling is off");
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < LMOSEM_K_COUNT; ++k) {
        h_ms[k] = 0.0;
        h_launches[k] = 0;
    }
    for (auto& r : c->prof) {
        float ms = 0.0f;
        LMOSEM_CK(c, cudaEventElapsedTime(&ms, r.a, r.b));
        h_ms[r.cls] += ms;
        h_launches[r.cls] += 1;
        c->prof_pool.push_back(r.a);
        c->prof_pool.push_back(r.b);
    }
    c->prof.clear();
    return LMOSEM_OK;
}

lmosem_status lmosem_model_rows(lmosem_ctx* c, const int64_t* d_ids, int64_t n, float* d_out) {
    if (!c) return LMOSEM_EINVAL;
    if (n < 0 || (n > 0 && (!d_ids || !d_out))) return fail(c, LMOSEM_EINVAL, "bad arguments");
    if (c->fmt < 0) return fail(c, LMOSEM_ESTATE, "no model built");
    return run_model_rows(c, d_ids, n, d_out);
}

lmosem_status lmosem_binned_support(lmosem_ctx* c, const int32_t* d_angle, const float* d_u_mm,
                                    const float* d_e_kev, int64_t n_events, int32_t n_subsets, int32_t n_iters,
                                    double threshold, int32_t dilate, uint8_t* h_support, float* d_image) {
    if (!c) return LMOSEM_EINVAL;
    if (!d_angle || !d_u_mm || !d_e_kev || !h_support) return fail(c, LMOSEM_EINVAL, "null argument");
    if (n_events < 1 || n_events >= (int64_t(1) << 31))
        return fail(c, LMOSEM_EINVAL, "n_events must be in [1, 2^31)");
    if (n_subsets < 1 || n_subsets > c->n_angles || n_iters < 1 || n_iters > 1000 || !(threshold > 0.0) ||
        !(threshold <= 1.0) || dilate < 0 || dilate > 8)
        return fail(c, LMOSEM_EINVAL,
                    "need 1 <= n_subsets <= n_angles, 1 <= n_iters <= 1000, 0 < threshold <= 1, 0 <= dilate <= 8");
    lmosem_status st = validate_events(c, d_angle, d_u_mm, d_e_kev, n_events);
    if (st) return st;
    return run_binned_support(c, d_angle, d_u_mm, n_events, n_subsets, n_iters, threshold, dilate, h_support,
                              d_image);
}

lmosem_status lmosem_surrogate_samples(lmosem_ctx* c, const int32_t* d_angle, const float* d_u_mm,
                                       const float* d_e_kev, int64_t n_events, float* d_features,
                                       float* d_log_scatter, float* d_rel_log) {
    if (!c) return LMOSEM_EINVAL;
    if (!d_features || !d_log_scatter) return fail(c, LMOSEM_EINVAL, "null output");
    lmosem_status st = check_events_args(c, d_angle, d_u_mm, d_e_kev, n_events, 1, LMOSEM_MODEL_FP32);
    if (st) return st;
    c->scatter_only = true;
    st = build_model_common(c, d_angle, d_u_mm, d_e_kev, n_events, 1, LMOSEM_MODEL_FP32, nullptr, 1);
    c->scatter_only = false;
    if (st) return st;
    st = run_surrogate_samples(c, d_features, d_log_scatter, d_rel_log);
    LMOSEM_CK(c, cudaStreamSynchronize(c->stream));
    free_model(c);
    return st;
}

lmosem_status lmosem_surrogate_train(lmosem_ctx* c, const float* d_features, const float* d_targets,
                                     const float* d_rel_log, int64_t n, const lmosem_train_opts* opts,
                                     float* d_weights, double* h_loss_curve) {
    if (!c) return LMOSEM_EINVAL;
    if (!d_features || !d_targets || !d_weights || !opts || n < 1)
        return fail(c, LMOSEM_EINVAL, "bad training arguments");
    if (opts->steps < 1 || opts->batch < 64 || opts->batch > 65536 || opts->batch % 64 ||
        !(opts->lr > 0.0f) || !isfinite(opts->lr) || !(opts->target_floor >= 0.0f) ||
        !isfinite(opts->target_floor))
        return fail(c, LMOSEM_EINVAL,
                    "steps >= 1, batch a multiple of 64 in [64, 65536], lr > 0, target_floor >= 0");
    if (opts->residual_fit != 0 && opts->residual_fit != 1) return fail(c, LMOSEM_EINVAL, "residual_fit is 0 or 1");
    if (!(opts->magnitude_power >= 0.0f) || !isfinite(opts->magnitude_power))
        return fail(c, LMOSEM_EINVAL, "magnitude_power must be finite and >= 0");
    return run_surrogate_train(c, d_features, d_targets, d_rel_log, n, opts->steps, opts->batch, opts->lr,
                               opts->seed, opts->target_floor, opts->residual_fit != 0, opts->magnitude_power,
                               d_weights, h_loss_curve);
}

lmosem_status lmosem_surrogate_grad(lmosem_ctx* c, const float* d_weights, const float* d_features,
                                    const float* d_targets, int64_t n, float* d_grad, double* h_loss) {
    if (!c) return LMOSEM_EINVAL;
    if (!d_weights || !d_features || !d_targets || !d_grad || n < 1 || n > 65536)
        return fail(c, LMOSEM_EINVAL, "bad gradient arguments (1 <= n <= 65536)");
    return run_surrogate_grad(c, d_weights, d_features, d_targets, n, d_grad, h_loss);
}

lmosem_status lmosem_surrogate_infer(lmosem_ctx* c, const float* d_weights, const float* d_features,
                                     int64_t n, float* d_out) {
    if (!c) return LMOSEM_EINVAL;
    if (!d_weights || !d_features || !d_out || n < 1 || n > (int64_t(1) << 26))
        return fail(c, LMOSEM_EINVAL, "bad inference arguments (1 <= n <= 2^26)");
    return run_surrogate_infer(c, d_weights, d_features, n, d_out);
}

lmosem_status lmosem_set_surrogate_check(lmosem_ctx* c, double tol, int32_t n_check_rows) {
    if (!c) return LMOSEM_EINVAL;
    if (!(tol >= 0.0) || !isfinite(tol) || n_check_rows < 0 || n_check_rows > 65536)
        return fail(c, LMOSEM_EINVAL, "need tol >= 0 (finite) and 0 <= n_check_rows <= 65536");
    c->sur_tol = tol;
    c->sur_check_rows = n_check_rows ? n_check_rows : 512;
    return LMOSEM_OK;
}

lmosem_status lmosem_surrogate_check(const lmosem_ctx* c, double* h_rel_err, double* h_row_max,
                                     int32_t* h_exact) {
    if (!c) return LMOSEM_EINVAL;
    if (!c->sur_checked) return LMOSEM_ESTATE;
    if (h_rel_err) *h_rel_err = c->sur_err;
    if (h_row_max) *h_row_max = c->sur_row_max;
    if (h_exact) *h_exact = c->sur_exact ? 1 : 0;
    return LMOSEM_OK;
}

lmosem_status lmosem_set_surrogate_gate(lmosem_ctx* c, double row_tol, double bin_kev) {
    if (!c) return LMOSEM_EINVAL;
    if (!(row_tol >= 0.0) || !isfinite(row_tol) || !(bin_kev >= 0.0) || !isfinite(bin_kev))
        return fail(c, LMOSEM_EINVAL, "need row_tol >= 0 and bin_kev >= 0 (finite)");
    c->sur_gate_tol = row_tol;
    c->sur_gate_bin = bin_kev > 0.0 ? bin_kev : 5.0;
    return LMOSEM_OK;
}

lmosem_status lmosem_surrogate_gate(const lmosem_ctx* c, double* h_e_cut_kev, double* h_frac_exact) {
    if (!c) return LMOSEM_EINVAL;
    if (!c->sur_checked) return LMOSEM_ESTATE;
    if (h_e_cut_kev) *h_e_cut_kev = c->sur_cut;
    if (h_frac_exact) *h_frac_exact = c->sur_frac_exact;
    return LMOSEM_OK;
}

lmosem_status lmosem_surrogate_load(lmosem_ctx* c, const float* d_weights) {
    if (!c) return LMOSEM_EINVAL;
    if (!d_weights) return fail(c, LMOSEM_EINVAL, "null weights");
    lmosem_status st;
    if (!c->d_surrogate && (st = dev_alloc(c, &c->d_surrogate, LMOSEM_SURROGATE_PARAMS))) return st;
    LMOSEM_CK(c, cudaMemcpyAsync(c->d_surrogate, d_weights, sizeof(float) * LMOSEM_SURROGATE_PARAMS,
                                 cudaMemcpyDeviceToDevice, c->stream));
    return LMOSEM_OK;
}

}  // extern "C"
