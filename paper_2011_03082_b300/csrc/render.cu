// ms_render / ms_render_batch (host side): request validation, the kernel variants and their autotuner, and the
// launch of the persistent render kernel (render_kernel.cuh) for sphere-traced (learned) and brute-force
// rendering of a homogeneous translucent SDF object with next-event estimation toward a point light.
#include "render_kernel.cuh"

using namespace ms::render;

// Compiled kernel variants (scheduling constants, MS_RENDER_VARIANTS): the FP32-decoder and brute-force
// instantiations live in this translation unit, the FP16 and BF16 ones in render_f16.cu and render_bf16.cu.
struct Variant {
    const void* fn;          // with the decoders in FP32 (any sphere-tracing request)
    const void* fn_brute;    // brute force only
    int decode_batch, trans_batch, steps, min_blocks;
};
#define MS_RENDER_ENTRY(d, t, s, m)                                                                            \
    Variant{(const void*)render_kernel<d, t, s, m, kDecFP32>, (const void*)render_kernel<d, t, s, m, kDecNone>, d, t,  \
            s, m},
static const Variant kVariants[] = {MS_RENDER_VARIANTS(MS_RENDER_ENTRY)};
#undef MS_RENDER_ENTRY
// The instrumented instantiations (phase timers) of the default variant.
static const void* const kTimedFP32 = (const void*)render_kernel<10, 12, 24, 3, kDecFP32, true>;
static const void* const kTimedBrute = (const void*)render_kernel<10, 12, 24, 3, kDecNone, true>;
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));

static ms_status fill_batch(const ms_render_params* reqs, int n, Batch* b, const char* fn)
{
    if (n < 1 || n > kMaxReq) return ms::set_error(MS_ERR_INVALID_ARG, "%s: 1..%d requests per call", fn, kMaxReq);
    if (reqs[0].variant < 0 || reqs[0].variant >= kNumVariants)
        return ms::set_error(MS_ERR_INVALID_ARG, "%s: variant must be in 0..%d", fn, kNumVariants - 1);
    uint64_t samples = 0, pixels = 0;
    b->n = n;
    for (int i = 0; i < n; ++i) {
        const ms_render_params& p = reqs[i];
        if (p.width < 1 || p.height < 1 || p.spp < 1)
            return ms::set_error(MS_ERR_INVALID_ARG, "%s: request %d: width, height and spp must be >= 1", fn, i);
        if (!(p.sigma_t > 0.0f) || !(p.g > -1.0f && p.g < 1.0f) || !(p.albedo >= 0.0f && p.albedo <= 1.0f))
            return ms::set_error(MS_ERR_INVALID_ARG, "%s: request %d: need sigma_t > 0, |g| < 1, albedo in [0,1]",
                                 fn, i);
        if (!(p.disp_amp >= 0.0f) || !(p.disp_freq >= 0.0f) || !(p.fov_y_deg > 0.0f && p.fov_y_deg < 180.0f))
            return ms::set_error(MS_ERR_INVALID_ARG, "%s: request %d: bad displacement or field of view", fn, i);
        if (p.mode != MS_BRUTE && p.mode != MS_SPHERE)
            return ms::set_error(MS_ERR_INVALID_ARG, "%s: request %d: mode must be MS_BRUTE or MS_SPHERE", fn, i);
        if (p.max_segments < 1) return ms::set_error(MS_ERR_INVALID_ARG, "%s: request %d: max_segments >= 1", fn, i);
        if ((uint64_t)p.width * p.height >= (1ull << 32) || p.sample_offset + p.spp > (1ull << 32))
            return ms::set_error(MS_ERR_INVALID_ARG, "%s: request %d: pixel or sample index exceeds 32 bits", fn, i);
        Req& q = b->r[i];
        for (int k = 0; k < 3; ++k) {
            q.cam[k] = p.cam_pos[k];
            q.at[k] = p.cam_at[k];
            q.light[k] = p.light_pos[k];
        }
        q.tan_half = (float)std::tan(0.5 * (double)p.fov_y_deg * 3.14159265358979323846 / 180.0);
        q.aspect = (float)p.width / (float)p.height;
        q.two_over_w = 2.0f / (float)p.width;
        q.two_over_h = 2.0f / (float)p.height;
        q.I = p.light_I;
        q.sigma = p.sigma_t;
        q.inv_sigma = 1.0f / p.sigma_t;
        q.din_cut = kTauCut / p.sigma_t;
        q.g = p.g;
        q.phi = p.albedo;
        q.log_phi = p.albedo > 0.0f ? std::log(p.albedo) : -INFINITY;
        q.A = p.disp_amp;
        q.k = p.disp_freq;
        q.lip = 1.0f + p.disp_amp * p.disp_freq;
        q.inv_lip = 1.0f / q.lip;
        const float rb = 1.0f + p.disp_amp + 1e-3f;
        q.rb2 = rb * rb;
        q.tau_min = p.min_optical_radius > 0.0f ? p.min_optical_radius
                                                 : ms_render_default_min_optical_radius(p.sigma_t);
        q.tau_max = p.max_optical_radius;
        if (p.sdf_grid != nullptr) {
            if (p.sdf_grid_n < 4 || p.sdf_grid_n > 1024 || !(p.disp_amp < 1.0f))
                return ms::set_error(MS_ERR_INVALID_ARG, "%s: request %d: sdf_grid_n must be in 4..1024", fn, i);
            const float h = 2.0f * (1.0f + p.disp_amp) / (float)(p.sdf_grid_n - 2);
            q.grid = p.sdf_grid;
            q.grid_n = p.sdf_grid_n;
            q.grid_b = 1.0f + p.disp_amp + h;
            q.grid_inv_h = 1.0f / h;
        } else {
            q.grid = nullptr;
            q.grid_n = 0;
            q.grid_b = q.grid_inv_h = 0.0f;
        }
        q.W = p.width;
        q.H = p.height;
        q.mode = p.mode;
        q.exact_n1 = p.exact_n1 != 0;
        q.exact_centre = p.exact_centre != 0;
        q.spp = p.spp;
        q.max_segments = p.max_segments;
        q.seed = p.seed;
        q.sample_offset = p.sample_offset;
        q.image_offset = pixels;
        q.samples_begin = samples;
        pixels += (uint64_t)p.width * p.height;
        samples += (uint64_t)p.width * p.height * p.spp;
    }
    b->total = samples;
    return MS_OK;
}

extern "C" size_t ms_render_workspace_size(const ms_render_params* reqs, int n_requests)
{
    (void)reqs;
    (void)n_requests;
    return 1024;   // ticket, start time, finished-path counters of up to 64 requests
}

static ms_status render_launch(const ms_render_params* reqs, int n, const ms_cvae_set* models, double* images,
                               unsigned long long* stats, void* workspace, size_t workspace_bytes, void* stream,
                               const char* fn)
{
    MS_CHECK_ARG(reqs != nullptr && images != nullptr && stats != nullptr, "%s: null argument", fn);
    const size_t need_ws = ms_render_workspace_size(reqs, n);
    MS_CHECK_ARG(workspace != nullptr && workspace_bytes >= need_ws && ((uintptr_t)workspace & 255u) == 0,
                 "%s: a 256-byte aligned workspace of at least %zu bytes is required", fn, need_ws);
    Batch b;
    ms_status st = fill_batch(reqs, n, &b, fn);
    if (st != MS_OK) return st;
    bool any_sphere = false;
    for (int i = 0; i < n; ++i) any_sphere |= reqs[i].mode == MS_SPHERE;
    b.wL = b.wP = b.wE = nullptr;
    int precision = MS_FP32;
    if (any_sphere) {
        MS_CHECK_ARG(models != nullptr, "%s: MS_SPHERE needs the three decoders", fn);
        const ms_decoder* d[3] = {&models->length, &models->path, &models->event};
        const int pin[3] = {2, 3, 7}, pout[3] = {1, 3, 6}, lat[3] = {kLatL, kLatP, kLatE}, wid[3] = {8, 16, 16};
        for (int k = 0; k < 3; ++k) {
            MS_CHECK_ARG(d[k]->weights != nullptr && d[k]->p_in == pin[k] && d[k]->p_out == pout[k] &&
                             d[k]->latent == lat[k] && d[k]->width == wid[k],
                         "%s: decoder %d must have p_in %d, latent %d, width %d, p_out %d (Table 1)", fn, k, pin[k],
                         lat[k], wid[k], pout[k]);
            MS_CHECK_ARG(d[k]->precision == MS_FP32 || d[k]->precision == MS_FP16 || d[k]->precision == MS_BF16,
                         "%s: decoder %d: precision must be MS_FP32, MS_FP16 or MS_BF16", fn, k);
            MS_CHECK_ARG(d[k]->precision == d[0]->precision, "%s: the three decoders must share one precision", fn);
        }
        precision = d[0]->precision;
        b.wL = models->length.weights;
        b.wP = models->path.weights;
        b.wE = models->event.weights;
    }
    b.image = images;
    b.stats = stats;
    b.ticket = static_cast<unsigned long long*>(workspace);
    b.t_start = b.ticket + 1;
    b.done = b.ticket + 2;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MS_CUDA(cudaMemsetAsync(workspace, 0, (2 + kMaxReq) * sizeof(unsigned long long), s));
    MS_CUDA(cudaMemsetAsync(b.t_start, 0xff, sizeof(unsigned long long), s));
    const Variant& v = kVariants[reqs[0].variant];
    if (reqs[0].phase_timers) {
        MS_CHECK_ARG(!any_sphere || precision == MS_FP32, "%s: phase timers need FP32 decoders", fn);
        MS_CHECK_ARG(kVariants[0].decode_batch == 10 && kVariants[0].trans_batch == 12 && kVariants[0].steps == 24,
                     "%s: the instrumented kernel is not the default variant's", fn);
    }
    const void* kfn = reqs[0].phase_timers ? (any_sphere ? kTimedFP32 : kTimedBrute)
                      : !any_sphere ? v.fn_brute
                      : precision == MS_FP16 ? variant_kernel_fp16(reqs[0].variant)
                      : precision == MS_BF16 ? variant_kernel_bf16(reqs[0].variant)
                                              : v.fn;
    MS_CHECK_ARG(kfn != nullptr, "%s: no kernel for variant %d", fn, reqs[0].variant);
    int per_sm = 0;
    MS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kThreads, 0));
    uint64_t grid = (uint64_t)ms::num_sms() * (per_sm > 0 ? per_sm : 1);
    const uint64_t need = (b.total + kThreads - 1) / kThreads;
    if (grid > need) grid = need;
    void* args[] = {&b};
    MS_CUDA(cudaLaunchKernel(kfn, dim3((unsigned)grid), dim3(kThreads), args, 0, s));
    return MS_OK;
}

extern "C" ms_status ms_render(const ms_render_params* p, const ms_cvae_set* models, double* image,
                               unsigned long long* stats, void* workspace, size_t workspace_bytes, void* stream)
{
    MS_NVTX("ms_render");
    return render_launch(p, 1, models, image, stats, workspace, workspace_bytes, stream, "ms_render");
}

extern "C" ms_status ms_render_batch(const ms_render_params* reqs, int n, const ms_cvae_set* models, double* images,
                                     unsigned long long* stats, void* workspace, size_t workspace_bytes,
                                     void* stream)
{
    MS_NVTX("ms_render_batch");
    return render_launch(reqs, n, models, images, stats, workspace, workspace_bytes, stream, "ms_render_batch");
}

extern "C" int ms_render_variants(void) { return kNumVariants; }

extern "C" ms_status ms_render_variant_info(int i, int* decode_batch, int* trans_batch, int* steps, int* min_blocks)
{
    MS_CHECK_ARG(i >= 0 && i < kNumVariants, "ms_render_variant_info: variant must be in 0..%d", kNumVariants - 1);
    if (decode_batch) *decode_batch = kVariants[i].decode_batch;
    if (trans_batch) *trans_batch = kVariants[i].trans_batch;
    if (steps) *steps = kVariants[i].steps;
    if (min_blocks) *min_blocks = kVariants[i].min_blocks;
    return MS_OK;
}

extern "C" ms_status ms_render_autotune(const ms_render_params* reqs, int n, const ms_cvae_set* models, double* images,
                                        unsigned long long* stats, void* workspace, size_t workspace_bytes,
                                        int repeats, int* best_variant, float* ms_per_variant, void* stream)
{
    MS_NVTX("ms_render_autotune");
    MS_CHECK_ARG(reqs != nullptr && n >= 1 && n <= kMaxReq && best_variant != nullptr,
                 "ms_render_autotune: need 1..%d requests and best_variant", kMaxReq);
    MS_CHECK_ARG(repeats >= 1, "ms_render_autotune: repeats must be >= 1");
    ms_render_params local[kMaxReq];
    for (int i = 0; i < n; ++i) local[i] = reqs[i];
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    MS_CUDA(cudaEventCreate(&e0));
    MS_CUDA(cudaEventCreate(&e1));
    float best = 0.0f;
    int best_i = -1;
    ms_status st = MS_OK;
    for (int v = 0; v < kNumVariants && st == MS_OK; ++v) {
        local[0].variant = v;
        st = render_launch(local, n, models, images, stats, workspace, workspace_bytes, stream, "ms_render_autotune");
        if (st != MS_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < repeats && st == MS_OK; ++r)
            st = render_launch(local, n, models, images, stats, workspace, workspace_bytes, stream, "ms_render_autotune");
        cudaEventRecord(e1, s);
        if (st != MS_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = ms::cuda_status(cudaGetLastError(), "ms_render_autotune: cudaEventSynchronize");
            break;
        }
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        t /= (float)repeats;
        if (ms_per_variant) ms_per_variant[v] = t;
        if (best_i < 0 || t < best) {
            best = t;
            best_i = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == MS_OK) *best_variant = best_i;
    return st;
}
