// Device-side records and per-ray arithmetic shared by the render and training kernels.
//
// Method: arXiv 2308.04669.  Ray transform to the object's canonical frame (Section
// "Manipulating Objects", Eq. 7), bound-sphere cull (Fig. 2b), tangency-point parametrisation
// (Eq. 2), sinusoidal input encodings, analytic object densities.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace nedf {

constexpr int kMaxLights = 32;
constexpr int kMaxTypes = 64;
constexpr int kNedfIn = 78;      // 6-D ray input, identity + 6 sin + 6 cos frequency blocks
constexpr int kNedfInPad = 80;   // padded to a multiple of 16 for tensor-core K steps
constexpr int kNerfIn = 90;      // 63 position features + 27 direction features
constexpr int kNerfInPad = 96;
constexpr uint32_t kNoId = 0xFFFFFFFFu;

// Device status bits (read back by nedf_compose_sync).
constexpr uint32_t kStatusPrimaryOverflow = 1u << 0;
constexpr uint32_t kStatusShadowOverflow = 1u << 1;
constexpr uint32_t kStatusTimeout = 1u << 2;
constexpr uint32_t kStatusResampleOverflow = 1u << 3;   // Step-2 resampling: more pairs than its buffers

struct DevType {
    int kind;
    float p[8];
    float rb;
    float albedo[3];
    int nerf;                 // 1 when a colour network exists
};

struct DevInst {              // 64 bytes
    float R[9];               // world = s R local + T
    float T[3];
    float s;
    uint32_t type;
    float pad[2];
};

struct DevFrame {
    float eye[3], right[3], up[3], fwd[3];
    float tan_h, aspect;
    int W, H;
    int n_lights;
    float lights[kMaxLights][3];       // point: position; parallel: unit travel direction
    uint32_t parallel_mask;            // bit l: light l is a parallel light
    // options
    int n_shade;
    float shade_half, beta, eps, sigma_max, sdf_width;
    int depth_source;
    int march_steps, march_bisect;
    float fallback_conf;
    int refine_steps;
    int outlier_resample;
    int shade_resample;          // Step-2 outlier resampling: plain-method samples per pair (0 = off)
    float shade_sigma_min;
    int miss_check;              // density samples that check a confident NeDF miss (0 = off)
    // buffer reuse while one instance is manipulated: 0 a whole frame; 1 the frozen part (every
    // instance but edit_inst); 2 an edit frame (the frozen buffers plus edit_inst alone)
    int edit_mode, edit_inst;
    int n_inst, n_types;
};

struct HostCamera {           // raw camera, turned into DevFrame's basis by a setup kernel
    float eye[3], target[3], fov_y_deg;
};

// ---------------------------------------------------------------------------------------------
// small vector helpers (explicit so both kernels that must agree compute identically)
// ---------------------------------------------------------------------------------------------
struct V3 { float x, y, z; };
__device__ __forceinline__ V3 v3(float x, float y, float z) { return V3{x, y, z}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 sub(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V3 madd(V3 a, float t, V3 d) { return v3(a.x + t * d.x, a.y + t * d.y, a.z + t * d.z); }
__device__ __forceinline__ V3 normalized(V3 a)
{
    float inv = 1.0f / sqrtf(dot(a, a));
    return v3(a.x * inv, a.y * inv, a.z * inv);
}

// Pinhole ray through the centre of pixel (i, j): u, v on the image plane at unit distance.
__device__ __forceinline__ void camera_ray(const DevFrame &f, int i, int j, V3 &o, V3 &d)
{
    float u = (2.0f * (i + 0.5f) / f.W - 1.0f) * f.tan_h * f.aspect;
    float v = (1.0f - 2.0f * (j + 0.5f) / f.H) * f.tan_h;
    o = v3(f.eye[0], f.eye[1], f.eye[2]);
    d = normalized(v3(u * f.right[0] + v * f.up[0] + f.fwd[0],
                      u * f.right[1] + v * f.up[1] + f.fwd[1],
                      u * f.right[2] + v * f.up[2] + f.fwd[2]));
}

// G^{-1} applied to a ray: local origin R^T (o - T) / s, local direction R^T d normalised.
// (R^T d / s normalised equals R^T d normalised; local lengths times s are world lengths.)
__device__ __forceinline__ void to_local(const DevInst &I, V3 o, V3 d, V3 &ol, V3 &dl)
{
    V3 v = sub(o, v3(I.T[0], I.T[1], I.T[2]));
    float is = 1.0f / I.s;
    ol = v3((I.R[0] * v.x + I.R[3] * v.y + I.R[6] * v.z) * is,
            (I.R[1] * v.x + I.R[4] * v.y + I.R[7] * v.z) * is,
            (I.R[2] * v.x + I.R[5] * v.y + I.R[8] * v.z) * is);
    dl = normalized(v3(I.R[0] * d.x + I.R[3] * d.y + I.R[6] * d.z,
                       I.R[1] * d.x + I.R[4] * d.y + I.R[7] * d.z,
                       I.R[2] * d.x + I.R[5] * d.y + I.R[8] * d.z));
}

struct Chord { float te, tx, tp; };

// Bound-sphere test of a unit local ray.  Kept iff the ray meets |x| = rb ahead of its origin.
// te = entry (clamped at the origin), tx = exit, tp = -o.d, the signed distance to the
// tangency point p_perp of Eq. 2.  The discriminant is rb^2 - |p_perp|^2 with p_perp formed
// explicitly, which avoids the cancellation of b^2 - (|o|^2 - rb^2) for distant origins.
__device__ __forceinline__ bool bound_chord(V3 ol, V3 dl, float rb, Chord &c)
{
    float b = dot(ol, dl);
    V3 pp = madd(ol, -b, dl);
    float disc = rb * rb - dot(pp, pp);
    c.tp = -b;
    if (disc < 0.0f) return false;
    float sq = sqrtf(disc);
    c.tx = -b + sq;
    c.te = fmaxf(0.0f, -b - sq);
    return c.tx >= 0.0f;
}

// ---------------------------------------------------------------------------------------------
// Analytic object shapes (object-local), density sigma = sigma_max / (1 + exp(sdf / w)).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float sdf_eval(const DevType &t, V3 x)
{
    const float *p = t.p;
    switch (t.kind) {
    case 0:  // sphere
        return sqrtf(dot(x, x)) - p[0];
    case 1: {  // torus, ring in the xz plane
        float q = sqrtf(x.x * x.x + x.z * x.z) - p[0];
        return sqrtf(q * q + x.y * x.y) - p[1];
    }
    case 2: {  // box
        float qx = fabsf(x.x) - p[0], qy = fabsf(x.y) - p[1], qz = fabsf(x.z) - p[2];
        float ox = fmaxf(qx, 0.f), oy = fmaxf(qy, 0.f), oz = fmaxf(qz, 0.f);
        return sqrtf(ox * ox + oy * oy + oz * oz) + fminf(fmaxf(qx, fmaxf(qy, qz)), 0.f);
    }
    case 3: {  // capsule along y
        float y = x.y - fminf(fmaxf(x.y, -p[0]), p[0]);
        return sqrtf(x.x * x.x + y * y + x.z * x.z) - p[1];
    }
    case 4: {  // rounded cone: hull of two spheres on the y axis
        float h = p[3] - p[1];
        float qr = sqrtf(x.x * x.x + x.z * x.z), qy = x.y - p[1];
        float sb = (p[0] - p[2]) / h, cb = sqrtf(1.0f - sb * sb);
        float k = -qr * sb + qy * cb;
        if (k < 0.0f) return sqrtf(qr * qr + qy * qy) - p[0];
        if (k > cb * h) return sqrtf(qr * qr + (qy - h) * (qy - h)) - p[2];
        return qr * cb + qy * sb - p[0];
    }
    case 5: {  // union of two spheres on the x axis
        float ax = x.x - p[0], bx = x.x + p[0], yz = x.y * x.y + x.z * x.z;
        return fminf(sqrtf(ax * ax + yz), sqrtf(bx * bx + yz)) - p[1];
    }
    case 6: {  // ring in the xy plane twisted about y
        float s, c;
        sincosf(p[2] * x.y, &s, &c);
        float xr = c * x.x - s * x.z, zr = s * x.x + c * x.z;
        float q = sqrtf(xr * xr + x.y * x.y) - p[0];
        return sqrtf(q * q + zr * zr) - p[1];
    }
    case 7:  // octahedron (distance lower bound)
        return (fabsf(x.x) + fabsf(x.y) + fabsf(x.z) - p[0]) * 0.57735026918962576f;
    default:
        return 1e30f;
    }
}

// Inside the solid <=> density >= sigma_max / 2 <=> sdf <= 0 (sigmoid(0) = 1/2).
__device__ __forceinline__ bool inside_solid(const DevType &t, V3 x) { return sdf_eval(t, x) <= 0.0f; }

// A Lipschitz bound of sdf_eval inside the bound sphere (|x| <= rb): the exact distances (sphere,
// torus, box, capsule, rounded cone), their minimum (two-sphere union) and the octahedron's lower
// bound have gradients of length <= 1; the twist by angle k y about the y axis stretches distances
// by at most sqrt(1 + (k rho)^2) <= 1 + |k| rb (rho: distance to the axis).
__device__ __forceinline__ float sdf_lipschitz(const DevType &t)
{
    return t.kind == 6 ? 1.0f + fabsf(t.p[2]) * t.rb : 1.0f;
}

// Samples within (|sdf(x)| - kSkipMargin) / Lipschitz of x along the ray lie on x's side of the
// surface.  The margin (local units) covers the FP32 error of the sample positions and of the SDF,
// so a skipped sample's own inside test could not have come out the other way.
constexpr float kSkipMargin = 1e-3f;

__device__ __forceinline__ float density(const DevType &t, V3 x, float sigma_max, float w)
{
    return sigma_max / (1.0f + expf(sdf_eval(t, x) / w));
}

// Plain method: steps uniform steps over [te, tx]; first outside -> inside step; bisection.
// Returns the crossing (local) or +inf.  Sample k is t_e + k (t_x - t_e) / steps, the step divided
// once (a division per sample would cost more than the density test it places).
__device__ __forceinline__ float march_crossing(const DevType &t, V3 ol, V3 dl, float te, float tx,
                                                int steps, int bisect, bool &hit)
{
    const float step = (tx - te) / (float)steps;
    float prev_t = te, kf = 0.0f;
    bool prev_in = inside_solid(t, madd(ol, te, dl));
    for (int k = 1; k <= steps; ++k) {
        kf += 1.0f;
        float tk = fmaf(kf, step, te);
        bool in = inside_solid(t, madd(ol, tk, dl));
        if (in && !prev_in) {
            float lo = prev_t, hi = tk;
            for (int it = 0; it < bisect; ++it) {
                float mid = 0.5f * (lo + hi);
                if (inside_solid(t, madd(ol, mid, dl))) hi = mid; else lo = mid;
            }
            hit = true;
            return 0.5f * (lo + hi);
        }
        prev_in = in;
        prev_t = tk;
    }
    hit = false;
    return __int_as_float(0x7f800000);
}

// march_crossing with the samples that the SDF proves to lie on the side of the last evaluated one
// skipped: the same first outside -> inside sample k, the same bracket [t_{k-1}, t_k] and the same
// bisection, so the same result, with a few SDF evaluations where a ray passes far from the surface
// instead of `steps`.
__device__ __forceinline__ float march_crossing_skip(const DevType &t, V3 ol, V3 dl, float te, float tx,
                                                     int steps, int bisect, bool &hit)
{
    const float step = (tx - te) / (float)steps;
    const float inv = 1.0f / (step * sdf_lipschitz(t));
    float sd = sdf_eval(t, madd(ol, te, dl));
    bool prev_in = sd <= 0.0f;
    int k = 0;
    while (true) {
        const float room = (fabsf(sd) - kSkipMargin) * inv;      // samples k+1 .. k+m keep k's side
        const int m = room > 0.0f ? (int)fminf(room, (float)steps) : 0;
        k += m + 1;
        if (k > steps) break;
        const float tk = fmaf((float)k, step, te);
        sd = sdf_eval(t, madd(ol, tk, dl));
        const bool in = sd <= 0.0f;
        if (in && !prev_in) {
            float lo = fmaf((float)(k - 1), step, te), hi = tk;
            for (int it = 0; it < bisect; ++it) {
                float mid = 0.5f * (lo + hi);
                if (inside_solid(t, madd(ol, mid, dl))) hi = mid; else lo = mid;
            }
            hit = true;
            return 0.5f * (lo + hi);
        }
        prev_in = in;
    }
    hit = false;
    return __int_as_float(0x7f800000);
}

// Bisection of the half-density level inside [D - h, D + h] when it brackets it.
__device__ __forceinline__ float refine_depth(const DevType &t, V3 ol, V3 dl, float D, float h, int steps)
{
    float lo = D - h, hi = D + h;
    if (inside_solid(t, madd(ol, lo, dl)) || !inside_solid(t, madd(ol, hi, dl))) return D;
    for (int it = 0; it < steps; ++it) {
        float mid = 0.5f * (lo + hi);
        if (inside_solid(t, madd(ol, mid, dl))) hi = mid; else lo = mid;
    }
    return 0.5f * (lo + hi);
}

// Decode of one NeDF answer (Eq. 2, Eq. 1's hit indicator) and the checks around it:
//   D_l = t_perp - rb * m, hit = (a > 0) and (D_l > 0);
//   a pair whose confidence max(p, 1 - p), p = sigmoid(a), is below fallback_conf goes to the
//   plain method; a hit whose window [D_l - h, D_l + h] brackets the half-density level is
//   refined by bisection there; a hit whose window does not is an outlier and, with
//   outlier_resample, also goes to the plain method; a miss that passed the confidence test is
//   checked at miss_check midpoints of the bound chord and goes to the plain method when the
//   density reaches the half level at one of them.
// Returns true when the pair must be re-answered by the plain method.
__device__ __forceinline__ bool nedf_decode(const DevFrame &f, const DevType &T, V3 ol, V3 dl, float tp, float m,
                                            float a, float &Dl, bool &hit)
{
    Dl = tp - T.rb * m;
    hit = (a > 0.0f) && (Dl > 0.0f);
    bool march = false;
    if (f.fallback_conf > 0.0f) {
        float p = 1.0f / (1.0f + expf(-a));
        march = fmaxf(p, 1.0f - p) < f.fallback_conf;
    }
    if (!march && !hit && f.miss_check > 0) {
        Chord ch;
        if (bound_chord(ol, dl, T.rb, ch)) {
            // the midpoints in order; samples the SDF proves outside are skipped (same answer)
            const float step = (ch.tx - ch.te) / (float)f.miss_check;
            const float inv = 1.0f / (step * sdf_lipschitz(T));
            for (int j = 0; j < f.miss_check;) {
                const float sd = sdf_eval(T, madd(ol, ch.te + ((float)j + 0.5f) * step, dl));
                if (sd <= 0.0f) {
                    march = true;
                    break;
                }
                const float room = (sd - kSkipMargin) * inv;
                j += 1 + (room > 0.0f ? (int)fminf(room, (float)f.miss_check) : 0);
            }
        }
    }
    if (!march && hit && f.refine_steps > 0) {
        float lo = Dl - f.shade_half, hi = Dl + f.shade_half;
        if (!inside_solid(T, madd(ol, lo, dl)) && inside_solid(T, madd(ol, hi, dl))) {
            for (int it = 0; it < f.refine_steps; ++it) {
                float mid = 0.5f * (lo + hi);
                if (inside_solid(T, madd(ol, mid, dl))) hi = mid; else lo = mid;
            }
            Dl = 0.5f * (lo + hi);
            hit = Dl > 0.0f;
        } else if (f.outlier_resample) {
            march = true;
        }
    }
    return march;
}

// ---------------------------------------------------------------------------------------------
// Counter-based SplitMix64 (Steele, Lea & Flood 2014): output `index` of the stream `seed`.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t index)
{
    uint64_t z = seed + (index + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float uniform24(uint64_t seed, uint64_t index)
{
    return (float)(uint32_t)(splitmix64_at(seed, index) >> 40) * (1.0f / 16777216.0f);
}

}  // namespace nedf
