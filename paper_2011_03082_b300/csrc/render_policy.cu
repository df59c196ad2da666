// ms_render_default_min_optical_radius: the renderer's thin-region fallback policy.  Kept apart from the render
// kernel so that retuning it leaves the kernel's translation unit unchanged.
#include <cmath>

#include "ms_device.cuh"

// The thin-region threshold per density (Sec. 6 names the fallback to path tracing where the sphere would be too
// thin): the minimum optical radius sigma_t r of a sphere step, below which a collision takes one brute-force
// event instead.  A larger threshold leaves more of the scattering near the surface, where the learned samplers
// are least accurate, to brute force, at a cost in time.  The knots are the thresholds of lowest time x squared
// error against a 16,384-spp brute-force reference, measured on the displaced-sphere scene at 512 x 512 px x
// 256 spp with the default model set (trained for the exact N = 1 step and centre event) over the thresholds
// 0.5, 1, 2, 4, 8; between knots the threshold is interpolated in log sigma_t, and held constant beyond the
// ends.  With that set the best threshold is 1 at every measured density (the set trained in the paper's
// form, whose small spheres are more biased, gave 0.5, 0.5, 1 and 2).
static const float kPolicySigma[] = {16.0f, 32.0f, 64.0f, 128.0f};
static const float kPolicyTau[] = {1.0f, 1.0f, 1.0f, 1.0f};
constexpr int kPolicyKnots = (int)(sizeof(kPolicySigma) / sizeof(kPolicySigma[0]));

extern "C" float ms_render_default_min_optical_radius(float sigma_t)
{
    if (!(sigma_t > kPolicySigma[0])) return kPolicyTau[0];
    for (int i = 1; i < kPolicyKnots; ++i)
        if (sigma_t <= kPolicySigma[i]) {
            const float t = std::log(sigma_t / kPolicySigma[i - 1]) / std::log(kPolicySigma[i] / kPolicySigma[i - 1]);
            return kPolicyTau[i - 1] + t * (kPolicyTau[i] - kPolicyTau[i - 1]);
        }
    return kPolicyTau[kPolicyKnots - 1];
}

