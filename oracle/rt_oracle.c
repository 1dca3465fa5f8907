/*
 * rt_oracle.c -- plain, slow FP64 CPU oracle of the per-pixel Whitted ray tracer of
 * "Accelerating Java Ray Tracing Applications on Heterogeneous Hardware"
 * (arXiv 2305.07450, Section 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * bench's CPU-baseline leg may load this library.  It shares no code, header,
 * table or constant with the CUDA path; both sides read the same FP32 scene
 * records (sphere [10], plane [10], light [8], camera [6]) and this side promotes
 * them to double before any arithmetic, so input rounding is not counted as error.
 *
 * Every function below follows one passage of the paper and says which.  Where the
 * paper is silent, ambiguous or garbled the reading taken is stated beside the code
 * (the same readings are listed in the design notes of the repository).
 *
 * Parity status: every function is pinned by a CPU test against something other
 * than itself (worked example, closed forms, invariants, brute force, published
 * known-answer vectors) -- see tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------ vectors */
typedef struct { double x, y, z; } v3;

static v3 V(double x, double y, double z) { v3 r; r.x = x; r.y = y; r.z = z; return r; }
static v3 add(v3 a, v3 b) { return V(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return V(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return V(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static double len(v3 a) { return sqrt(dot(a, a)); }
static v3 nrm(v3 a) { return scl(a, 1.0 / len(a)); }

/* ------------------------------------------------------------------- inputs */
/* Public input block, filled by the Python wrapper (ctypes).  Field order is the
 * oracle's own; it is not the device library's rt_scene_desc. */
typedef struct {
    int n_spheres;
    const float *spheres;   /* [n][10] cx cy cz r  ar ag ab  ks exp refl           */
    int has_plane;
    const float *plane;     /* [10]    nx ny nz d  ar ag ab  ks exp refl           */
    int n_lights;
    const float *lights;    /* [L][8]  x y z I  area_side sphere_radius 0 0       */
    const float *camera;    /* [6]     x y z yaw_deg pitch_deg fov_deg            */
    int width, height;
    int max_depth;          /* reflection bounce limit D                          */
    int shadow_samples;     /* samples per sampled light                           */
    int shading_model;      /* 0 Phong, 1 Blinn-Phong                              */
    int pad_;
    double ambient;         /* k_a                                                 */
    double eps;             /* absolute offset of secondary ray origins            */
    double scene_scale;     /* length unit of the margins                          */
    uint64_t seed;          /* Philox key                                          */
    int refl_coupled;       /* 1: reflection ratio = spec_exp / max_reflectivity   */
    int pad2_;
    double max_reflectivity;
    const float *sky;       /* [sky_h][sky_w][4] RGBA panorama, or NULL (black)    */
    int sky_w, sky_h;
} orc_in;

/* One primitive promoted to FP64.  For the plane, g = normal and r = d. */
typedef struct { v3 g; double r; double alb[3]; double ks, ex, rho; } Prim;
typedef struct { v3 p; double I, area, srad; } Light;

enum {
    C_PRIMARY = 0, C_REFLECT, C_SHADOW, C_CLOSEST_SPH, C_CLOSEST_PLANE,
    C_SHADOW_SPH, C_SHADOW_PLANE, C_HITS, C_LIT, C_SAMPLES, C_PHILOX, C_NCOUNT = 12
};

typedef struct {
    int ns, np;             /* spheres, 1 if plane */
    Prim *prim;             /* ns spheres then the plane */
    int nl;
    Light *light;
    v3 cam;
    double yaw, pitch, fov; /* radians */
    int W, H, D, nsamp, model;
    double ka, eps, S;
    uint32_t key[2];
    const float *sky;
    int sky_w, sky_h;
} Ctx;

typedef struct {
    const Ctx *cx;
    int want_margin;
    double margin;
    double cnt[C_NCOUNT];
    uint32_t pix;           /* y * W + x, the Philox counter word 0 */
    int origin;             /* primitive the current ray leaves (-1: the camera) */
} Path;

/* ------------------------------------------------------------ Philox4x32-10 */
/* Counter-based generator of Salmon, Moraes, Dror and Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64 multiplies,
 * an xor with the round key and a word permutation; the key is bumped by the two
 * Weyl constants between rounds. */
static void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 24 high bits of a word as a uniform in [0, 1): exact in FP32 and FP64. */
static double u01(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------- camera, Sections 3.2-3.3 */
/* Section 3.2, NDC listing: the shorter image side spans [-1, 1].  Reading: pixel
 * coordinates are the integer x, y with no half-pixel shift (the worked example of
 * Section 3.3.1 maps (640, 360) of 1280x720 to (0, 0)), and width/2, height/2 are
 * real divisions. */
static void ndc(int W, int H, double x, double y, double *u, double *v)
{
    double w = W, h = H;
    if (w > h) {
        *u = (x - w / 2.0 + h / 2.0) / h * 2.0 - 1.0;
        *v = -(y / h * 2.0 - 1.0);
    } else {
        *u = x / w * 2.0 - 1.0;
        *v = -((y - h / 2.0 + w / 2.0) / w * 2.0 - 1.0);
    }
}

/* Section 3.2.1: half viewport side a = 1, so b = a / tan(alpha / 2). */
static double camera_distance(double fov_rad) { return 1.0 / tan(fov_rad / 2.0); }

/* Section 3.3.1: P = (u, v, 0), C = (0, 0, -b), direction = normalize(P - C) (the
 * text's "P subtracted from C" would point backwards; reading: P - C, forward is
 * +z), then rotated by the camera's pitch (about x, positive looks up) and then its
 * yaw (about y, positive turns toward +x); origin = camera position. */
static void primary_ray(const Ctx *cx, double x, double y, double du, double dv, v3 *o, v3 *d)
{
    double u, v;
    ndc(cx->W, cx->H, x, y, &u, &v);
    u += du;
    v += dv;
    double b = camera_distance(cx->fov);
    v3 P = V(u, v, 0.0), C = V(0.0, 0.0, -b);
    v3 r = nrm(sub(P, C));
    double cp = cos(cx->pitch), sp = sin(cx->pitch);
    r = V(r.x, r.y * cp + r.z * sp, -r.y * sp + r.z * cp);
    double cyw = cos(cx->yaw), syw = sin(cx->yaw);
    r = V(r.x * cyw + r.z * syw, r.y, -r.x * syw + r.z * cyw);
    *o = cx->cam;
    *d = r;
}

/* ------------------------------------------------ intersections, Section 3.4 */
/* Ray-sphere (Section 3.4, "Size" is the radius): roots of |o + t d - c|^2 = r^2
 * for a unit d.  Returns the near root if it is > 0, else the far root if > 0
 * (a tangent ray, disc = 0, counts as a hit). */
static int sphere_root(v3 o, v3 d, v3 c, double r, double *t)
{
    v3 oc = sub(o, c);
    double b = dot(oc, d);
    double q = dot(oc, oc) - r * r;
    double disc = b * b - q;
    if (disc < 0.0) return 0;
    double s = sqrt(disc);
    double tn = -b - s;
    if (tn > 0.0) { *t = tn; return 1; }
    double tf = -b + s;
    if (tf > 0.0) { *t = tf; return 1; }
    return 0;
}

/* Ray-plane n.x + d = 0 (the paper's ground plane; reading: infinite, two-sided). */
static int plane_root(v3 o, v3 dir, v3 n, double pd, double *t)
{
    double den = dot(dir, n);
    if (den == 0.0) return 0;
    double tt = -(dot(o, n) + pd) / den;
    if (tt > 0.0) { *t = tt; return 1; }
    return 0;
}

/* Margin of one closest-hit ray (length units): sphere silhouettes that could
 * compete with the hit, roots near the origin, the gap to the second-nearest
 * primitive, and the plane's horizon when the plane wins or nothing is hit.  The
 * primitive the ray leaves (P->origin) has no root near the origin by
 * construction (the origin is offset along its normal, so its roots lie at or
 * behind -eps), and is skipped in that term. */
static void closest_margin(Path *P, v3 o, v3 d, int best, double tb)
{
    const Ctx *cx = P->cx;
    double m = INFINITY, t2 = INFINITY;
    for (int i = 0; i < cx->ns; ++i) {
        const Prim *s = &cx->prim[i];
        v3 oc = sub(s->g, o);
        double tca = dot(oc, d);
        double ld = len(sub(oc, scl(d, tca)));
        if (tca + s->r > 0.0 && (best < 0 || tca - s->r < tb)) m = fmin(m, fabs(ld - s->r));
        double disc = s->r * s->r - ld * ld;
        if (disc >= 0.0 && i != P->origin) {
            double sq = sqrt(disc);
            m = fmin(m, fabs(tca - sq));
            m = fmin(m, fabs(tca + sq));
        }
        double t;
        if (i != best && sphere_root(o, d, s->g, s->r, &t)) t2 = fmin(t2, t);
    }
    if (cx->np) {
        const Prim *pl = &cx->prim[cx->ns];
        double den = dot(d, pl->g);
        if (best == cx->ns || best < 0) m = fmin(m, fabs(den) * cx->S);
        if (den != 0.0) {
            double tp = -(dot(o, pl->g) + pl->r) / den;
            if (P->origin != cx->ns) m = fmin(m, fabs(tp));
            if (best != cx->ns && tp > 0.0) t2 = fmin(t2, tp);
        }
    }
    if (best >= 0 && t2 < INFINITY) m = fmin(m, t2 - tb);
    P->margin = fmin(P->margin, m);
}

/* Section 3.4.1: check the ray against every object (brute force, no acceleration
 * structure) and keep the closest.  Reading: strict '<', so on equal distances the
 * lowest index wins; spheres are 0..N-1 and the plane is N.  Returns -1 on a miss. */
static int closest_hit(Path *P, v3 o, v3 d, double *t_out)
{
    const Ctx *cx = P->cx;
    int best = -1;
    double tb = INFINITY, t;
    for (int i = 0; i < cx->ns; ++i) {
        P->cnt[C_CLOSEST_SPH] += 1;
        if (sphere_root(o, d, cx->prim[i].g, cx->prim[i].r, &t) && t < tb) { tb = t; best = i; }
    }
    if (cx->np) {
        P->cnt[C_CLOSEST_PLANE] += 1;
        const Prim *pl = &cx->prim[cx->ns];
        if (plane_root(o, d, pl->g, pl->r, &t) && t < tb) { tb = t; best = cx->ns; }
    }
    if (P->want_margin) closest_margin(P, o, d, best, tb);
    *t_out = tb;
    return best;
}

/* Section 3.6, cast-shadows listing: a shadow ray from the surface toward the light
 * is blocked if any object is hit closer than the light; the loop stops at the first
 * blocker.  Reading: every primitive is tested (the hit's own one included: it can
 * never block, since a ray is only cast when n.l > 0 and the origin is offset along
 * n); a root must lie in (0, dist). */
static int occluded(Path *P, v3 o, v3 dir, double dist)
{
    const Ctx *cx = P->cx;
    P->cnt[C_SHADOW] += 1;
    double m = INFINITY;
    int hit = 0;
    for (int i = 0; i < cx->ns && !hit; ++i) {
        const Prim *s = &cx->prim[i];
        P->cnt[C_SHADOW_SPH] += 1;
        double t;
        if (sphere_root(o, dir, s->g, s->r, &t) && t < dist) hit = 1;
        if (P->want_margin) {
            v3 oc = sub(s->g, o);
            double tca = dot(oc, dir);
            double ld = len(sub(oc, scl(dir, tca)));
            if (tca >= 0.0 && tca <= dist) m = fmin(m, fabs(ld - s->r));
            double disc = s->r * s->r - ld * ld;
            if (disc >= 0.0) {
                double sq = sqrt(disc);
                double r1 = tca - sq, r2 = tca + sq;
                m = fmin(m, fabs(r1 - dist));
                m = fmin(m, fabs(r2 - dist));
                if (i != P->origin) m = fmin(m, fmin(fabs(r1), fabs(r2)));
            }
        }
    }
    if (!hit && cx->np) {
        const Prim *pl = &cx->prim[cx->ns];
        P->cnt[C_SHADOW_PLANE] += 1;
        double t;
        if (plane_root(o, dir, pl->g, pl->r, &t) && t < dist) hit = 1;
        if (P->want_margin) {
            double den = dot(dir, pl->g);
            if (den != 0.0) {
                double tp = -(dot(o, pl->g) + pl->r) / den;
                m = fmin(m, fabs(tp - dist));
                if (P->origin != cx->ns) m = fmin(m, fabs(tp));
            }
        }
    }
    if (P->want_margin) P->margin = fmin(P->margin, m);
    return hit;
}

#define ORC_MAX_SAMPLES 4096

/* Sample points of a square area light (a stand-in for the paper's soft shadows of
 * Section 3.6.1, which multiply the light by a shadow coefficient in [0, 1]): side a,
 * horizontal, centred on the light position; n = g*g strata in a g x g grid, one
 * sample per stratum at ((i + xi1)/g - 1/2, (j + xi2)/g - 1/2) * a in x and z.
 * Sample s uses stratum (s mod g, s div g) and Philox call s div 2 with counter
 * (pixel, bounce, light, call), words 2(s mod 2) and 2(s mod 2) + 1. */
static int area_samples(const Ctx *cx, uint32_t pix, int k, int l, v3 *pts, double *philox_calls)
{
    const Light *L = &cx->light[l];
    int g = (int)lround(sqrt((double)cx->nsamp));
    int n = g * g;
    uint32_t words[4] = {0, 0, 0, 0};
    for (int s = 0; s < n; ++s) {
        if ((s & 1) == 0) {
            uint32_t ctr[4] = {pix, (uint32_t)k, (uint32_t)l, (uint32_t)(s >> 1)};
            philox4x32_10(ctr, cx->key, words);
            if (philox_calls) *philox_calls += 1;
        }
        double xi1 = u01(words[2 * (s & 1)]), xi2 = u01(words[2 * (s & 1) + 1]);
        int i = s % g, j = s / g;
        pts[s] = add(L->p, V(((i + xi1) / g - 0.5) * L->area, 0.0, ((j + xi2) / g - 0.5) * L->area));
    }
    return n;
}

/* Sample points of a spherical light of radius R, Section 3.6.1: n points of the
 * sunflower (Vogel) arrangement on the great circle of the light that faces the
 * point p, r(i) = R sqrt(i / n), theta(i) = i * phi, phi = pi (3 - sqrt 5).
 * Reading: the printed "2 x radius" would put points outside the circle, so the
 * disc radius is the light radius; the circle's in-plane axes are
 * u = normalize(w x up) and v = u x w, w = unit vector from the light to p,
 * up = +y (or +x when w is nearly vertical). */
static int vogel_samples(const Ctx *cx, int l, v3 p, v3 *pts)
{
    const Light *L = &cx->light[l];
    int n = cx->nsamp;
    v3 w = nrm(sub(p, L->p));
    v3 up = fabs(w.y) < 0.999 ? V(0.0, 1.0, 0.0) : V(1.0, 0.0, 0.0);
    v3 u = nrm(V(w.y * up.z - w.z * up.y, w.z * up.x - w.x * up.z, w.x * up.y - w.y * up.x));
    v3 v = V(u.y * w.z - u.z * w.y, u.z * w.x - u.x * w.z, u.x * w.y - u.y * w.x);
    double phi = M_PI * (3.0 - sqrt(5.0));
    for (int i = 0; i < n; ++i) {
        double r = L->srad * sqrt((double)i / (double)n);
        double th = i * phi;
        pts[i] = add(L->p, add(scl(u, r * cos(th)), scl(v, r * sin(th))));
    }
    return n;
}

/* Visible fraction of a sampled light: one shadow ray from the offset origin toward
 * each sample point, as far as that point; the fraction of unblocked rays is the
 * paper's shadow coefficient (Section 3.6.1). */
static double sampled_visibility(Path *P, int k, int l, v3 p, v3 po)
{
    const Ctx *cx = P->cx;
    v3 pts[ORC_MAX_SAMPLES];
    int n = cx->light[l].area > 0.0 ? area_samples(cx, P->pix, k, l, pts, &P->cnt[C_PHILOX])
                                    : vogel_samples(cx, l, p, pts);
    int unblocked = 0;
    for (int s = 0; s < n; ++s) {
        v3 to = sub(pts[s], p);
        double dist = len(to);
        P->cnt[C_SAMPLES] += 1;
        if (!occluded(P, po, scl(to, 1.0 / dist), dist)) unblocked += 1;
    }
    return (double)unblocked / (double)n;
}

static double powpos(double x, double e) { return x > 0.0 ? pow(x, e) : 0.0; }

/* Section 3.5 (Phong, ambient / diffuse / specular), Section 3.5.2 (Blinn) and
 * Section 3.6 (shadows).  shade(c) is affine in the colour c it is given:
 *     shade(c) = c * A + S,
 *     A = k_a + sum_l I_l vis_l max(n.l, 0),
 *     S = sum_l I_l vis_l k_s spec_l.
 * Readings (the paper prints no combination formula): white lights of intensity
 * I_l, no distance attenuation; a light is skipped when n.l <= 0 (no diffuse, no
 * specular, no shadow ray); a shadowed light leaves only the ambient share, as the
 * paper states for cast shadows.  Phong: spec = max(v.r, 0)^exp with r the light
 * direction mirrored about n and v = -d (the listing's camera-minus-surface for a
 * primary ray).  Blinn: spec = max(n.h, 0)^exp, h = normalize(l + v).  The shadow
 * ray of a point light leaves from p + eps n along l for distance |L - p|. */
static void shade_terms(Path *P, int k, v3 p, v3 n, v3 d, const Prim *m, double *A, double *S)
{
    const Ctx *cx = P->cx;
    v3 po = add(p, scl(n, cx->eps));
    v3 view = scl(d, -1.0);
    double a = cx->ka, s = 0.0;
    P->cnt[C_HITS] += 1;
    for (int l = 0; l < cx->nl; ++l) {
        const Light *L = &cx->light[l];
        v3 to = sub(L->p, p);
        double dist = len(to);
        v3 lh = scl(to, 1.0 / dist);
        double ndl = dot(n, lh);
        if (P->want_margin) P->margin = fmin(P->margin, fabs(ndl) * cx->S);
        if (ndl <= 0.0) continue;
        P->cnt[C_LIT] += 1;
        double vis;
        if (L->area > 0.0 || L->srad > 0.0) vis = sampled_visibility(P, k, l, p, po);
        else vis = occluded(P, po, lh, dist) ? 0.0 : 1.0;
        double sp;
        if (cx->model == 0) {
            v3 r = sub(scl(n, 2.0 * ndl), lh);
            sp = powpos(dot(view, r), m->ex);
        } else {
            v3 h = nrm(add(lh, view));
            sp = powpos(dot(n, h), m->ex);
        }
        a += L->I * vis * ndl;
        s += L->I * vis * m->ks * sp;
    }
    *A = a;
    *S = s;
}

/* Geometry at a hit: point and unit normal, face-forwarded (reading: flipped to
 * face the incoming ray).  Sphere: the unit vector from the centre through the
 * hit point, normalize(p - c) -- equal to (p - c)/r on the surface; evaluated as
 * a normalisation so that the rounding of the root cannot make |n| differ from 1
 * (the reflection below keeps |d| = 1 only for a unit n, and the root formula
 * assumes a unit d).  Plane: its unit normal. */
static void hit_geometry(const Ctx *cx, int id, v3 o, v3 d, double t, v3 *p, v3 *n)
{
    *p = add(o, scl(d, t));
    if (id < cx->ns) *n = nrm(sub(*p, cx->prim[id].g));
    else *n = cx->prim[id].g;
    if (dot(*n, d) > 0.0) *n = scl(*n, -1.0);
}

/* --------------------------------------------------------------- Section 3.8 sky */
/* A ray that leaves the scene shows the sky: the paper samples an HDR panorama by
 * UV mapping of the ray direction (Section 3.8, skybox; Section 3.9 skybox
 * argument).  Reading: an equirectangular panorama of W x H RGBA texels stored
 * row-major from the top row, with the spherical UV mapping of a unit direction
 *   u = 1/2 + atan2(d_z, d_x) / (2 pi),   v = 1/2 - asin(d_y) / pi,
 * and bilinear interpolation between texel centres ((i + 1/2) / W, (j + 1/2) / H),
 * wrapping around in u and clamped to the first and last rows in v. */
static double sky_texel(const float *tex, int W, int i, int j, int c) { return tex[((size_t)j * W + i) * 4 + c]; }

static void sky_lookup(const float *tex, int W, int H, v3 d, double out[3])
{
    const double dy = fmax(-1.0, fmin(1.0, d.y / len(d)));
    const double u = 0.5 + atan2(d.z, d.x) / (2.0 * M_PI);
    const double v = 0.5 - asin(dy) / M_PI;
    const double x = u * W - 0.5, y = v * H - 0.5;
    const double x0 = floor(x), y0 = floor(y);
    const double fx = x - x0, fy = y - y0;
    int i0 = (int)fmod(x0, (double)W);
    if (i0 < 0) i0 += W;
    const int i1 = (i0 + 1) % W;
    int j0 = (int)y0, j1 = (int)y0 + 1;
    j0 = j0 < 0 ? 0 : (j0 > H - 1 ? H - 1 : j0);
    j1 = j1 < 0 ? 0 : (j1 > H - 1 ? H - 1 : j1);
    for (int c = 0; c < 3; ++c) {
        const double top = (1.0 - fx) * sky_texel(tex, W, i0, j0, c) + fx * sky_texel(tex, W, i1, j0, c);
        const double bot = (1.0 - fx) * sky_texel(tex, W, i0, j1, c) + fx * sky_texel(tex, W, i1, j1, c);
        out[c] = (1.0 - fy) * top + fy * bot;
    }
}

static void miss_color(const Ctx *cx, v3 d, double out[3])
{
    if (cx->sky) sky_lookup(cx->sky, cx->sky_w, cx->sky_h, d, out);
    else out[0] = out[1] = out[2] = 0.0;
}

/* Section 3.7.1, recursive reflections, written literally: a miss is black (or the
 * sky, Section 3.8, when one is given); at the bounce limit the hit is shaded with its own colour; otherwise the colour is mixed
 * with the reflected colour by the reflection ratio and the mix is shaded.  The
 * reflection ratio is the per-object reflectivity field (reading: the paper derives
 * it as reflectivity / MAX_REFLECTIVITY with the same field as the Phong exponent;
 * here exponent and ratio are separate fields).  `depth` counts down as in the
 * paper; k = D - depth is the bounce index. */
static void trace_recursive(Path *P, v3 o, v3 d, int depth, int k, int origin, double out[3])
{
    const Ctx *cx = P->cx;
    P->cnt[k == 0 ? C_PRIMARY : C_REFLECT] += 1;
    double t;
    P->origin = origin;
    int id = closest_hit(P, o, d, &t);
    if (id < 0) { miss_color(cx, d, out); return; }
    const Prim *m = &cx->prim[id];
    v3 p, n;
    hit_geometry(cx, id, o, d, t, &p, &n);
    double col[3];
    if (depth == 0) {
        col[0] = m->alb[0]; col[1] = m->alb[1]; col[2] = m->alb[2];
    } else {
        v3 rd = sub(d, scl(n, 2.0 * dot(d, n)));
        v3 ro = add(p, scl(n, cx->eps));
        double rc[3];
        trace_recursive(P, ro, rd, depth - 1, k + 1, id, rc);
        for (int c = 0; c < 3; ++c) col[c] = m->alb[c] * (1.0 - m->rho) + rc[c] * m->rho;
    }
    double A, S;
    P->origin = id;
    shade_terms(P, k, p, n, d, m, &A, &S);
    for (int c = 0; c < 3; ++c) out[c] = col[c] * A + S;
}

/* The same definition unrolled forward (Section 3.7.2 replaces the recursion by a
 * loop).  Since shade(c) = c A + S is affine, with throughput T_0 = 1:
 *   k < D : out += T_k ((1 - rho_k) A_k c_k + S_k),  T_{k+1} = T_k rho_k A_k
 *   k = D : out += T_D (A_D c_D + S_D);  a miss at bounce k adds T_k sky(d_k) (nothing
 *   without a sky) and ends the path. */
static void trace_forward(Path *P, v3 o, v3 d, double out[3])
{
    const Ctx *cx = P->cx;
    double T = 1.0;
    out[0] = out[1] = out[2] = 0.0;
    P->origin = -1;
    for (int k = 0; k <= cx->D; ++k) {
        P->cnt[k == 0 ? C_PRIMARY : C_REFLECT] += 1;
        double t;
        int id = closest_hit(P, o, d, &t);
        if (id < 0) {
            double sk[3];
            miss_color(cx, d, sk);
            for (int c = 0; c < 3; ++c) out[c] += T * sk[c];
            break;
        }
        P->origin = id;
        const Prim *m = &cx->prim[id];
        v3 p, n;
        hit_geometry(cx, id, o, d, t, &p, &n);
        double A, S;
        shade_terms(P, k, p, n, d, m, &A, &S);
        if (k < cx->D) {
            for (int c = 0; c < 3; ++c) out[c] += T * ((1.0 - m->rho) * A * m->alb[c] + S);
            T *= m->rho * A;
            d = sub(d, scl(n, 2.0 * dot(d, n)));
            o = add(p, scl(n, cx->eps));
        } else {
            for (int c = 0; c < 3; ++c) out[c] += T * (A * m->alb[c] + S);
        }
    }
}

/* -------------------------------------------------------------- entry points */
static int build_ctx(const orc_in *in, Ctx *cx)
{
    if (!in || in->width <= 0 || in->height <= 0 || in->max_depth < 0 || in->n_spheres < 0
        || (in->refl_coupled && !(in->max_reflectivity > 0.0))
        || in->n_lights < 0 || !in->camera || (in->n_spheres && !in->spheres)
        || (in->n_lights && !in->lights) || (in->has_plane && !in->plane))
        return -1;
    memset(cx, 0, sizeof(*cx));
    cx->ns = in->n_spheres;
    cx->np = in->has_plane ? 1 : 0;
    cx->nl = in->n_lights;
    cx->prim = (Prim *)calloc((size_t)(cx->ns + cx->np + 1), sizeof(Prim));
    cx->light = (Light *)calloc((size_t)(cx->nl + 1), sizeof(Light));
    if (!cx->prim || !cx->light) { free(cx->prim); free(cx->light); return -2; }
    for (int i = 0; i < cx->ns + cx->np; ++i) {
        const float *f = i < cx->ns ? in->spheres + 10 * i : in->plane;
        Prim *p = &cx->prim[i];
        p->g = V(f[0], f[1], f[2]);
        p->r = f[3];
        p->alb[0] = f[4]; p->alb[1] = f[5]; p->alb[2] = f[6];
        p->ks = f[7]; p->ex = f[8]; p->rho = f[9];
        /* Section 3.7: the paper derives the reflection ratio from the same
         * reflectivity value that is the Phong exponent, divided by
         * MAX_REFLECTIVITY (a fully reflective mirror at the maximum). */
        if (in->refl_coupled) p->rho = fmin(p->ex / in->max_reflectivity, 1.0);
    }
    int sampled = 0;
    for (int l = 0; l < cx->nl; ++l) {
        const float *f = in->lights + 8 * l;
        cx->light[l].p = V(f[0], f[1], f[2]);
        cx->light[l].I = f[3];
        cx->light[l].area = f[4];
        cx->light[l].srad = f[5];
        if (f[4] > 0.0f || f[5] > 0.0f) sampled = 1;
        if (f[4] > 0.0f && f[5] > 0.0f) { free(cx->prim); free(cx->light); return -1; }
    }
    cx->nsamp = in->shadow_samples;
    if (sampled) {
        int g = (int)lround(sqrt((double)cx->nsamp));
        if (cx->nsamp <= 0 || cx->nsamp > ORC_MAX_SAMPLES) { free(cx->prim); free(cx->light); return -1; }
        for (int l = 0; l < cx->nl; ++l)
            if (cx->light[l].area > 0.0 && g * g != cx->nsamp) {
                free(cx->prim); free(cx->light); return -1;
            }
    }
    const double deg = M_PI / 180.0;
    cx->cam = V(in->camera[0], in->camera[1], in->camera[2]);
    cx->yaw = in->camera[3] * deg;
    cx->pitch = in->camera[4] * deg;
    cx->fov = in->camera[5] * deg;
    cx->W = in->width;
    cx->H = in->height;
    cx->D = in->max_depth;
    cx->model = in->shading_model;
    cx->ka = in->ambient;
    cx->eps = in->eps;
    cx->S = in->scene_scale;
    cx->key[0] = (uint32_t)(in->seed & 0xffffffffu);
    cx->key[1] = (uint32_t)(in->seed >> 32);
    if (in->sky && (in->sky_w <= 0 || in->sky_h <= 0)) { free(cx->prim); free(cx->light); return -1; }
    cx->sky = in->sky;
    cx->sky_w = in->sky_w;
    cx->sky_h = in->sky_h;
    return 0;
}

/* Trace n pixels (xy = int32 pairs x, y).  mode 0 = forward form, 1 = literal
 * recursion.  (du, dv) shifts every pixel's NDC (0, 0 for the definition).
 * rgb: [n][3] linear colour, not clamped.  margin (nullable): [n] minimum margin
 * over the pixel's whole path.  counters (nullable): [12], accumulated.
 * Returns 0, or -1 for invalid input, -2 when out of memory. */
ORC_API int orc_trace(const orc_in *in, int mode, int n, const int32_t *xy, double du, double dv,
                      double *rgb, double *margin, double *counters)
{
    Ctx cx;
    int st = build_ctx(in, &cx);
    if (st) return st;
    if (n < 0 || (n && (!xy || !rgb))) { free(cx.prim); free(cx.light); return -1; }
    Path P;
    memset(&P, 0, sizeof(P));
    P.cx = &cx;
    P.want_margin = margin != NULL;
    for (int i = 0; i < n; ++i) {
        int x = xy[2 * i], y = xy[2 * i + 1];
        if (x < 0 || y < 0 || x >= cx.W || y >= cx.H) { free(cx.prim); free(cx.light); return -1; }
        P.pix = (uint32_t)y * (uint32_t)cx.W + (uint32_t)x;
        P.margin = INFINITY;
        v3 o, d;
        primary_ray(&cx, x, y, du, dv, &o, &d);
        if (mode == 1) trace_recursive(&P, o, d, cx.D, 0, -1, rgb + 3 * i);
        else trace_forward(&P, o, d, rgb + 3 * i);
        if (margin) margin[i] = P.margin;
    }
    if (counters)
        for (int c = 0; c < C_NCOUNT; ++c) counters[c] += P.cnt[c];
    free(cx.prim);
    free(cx.light);
    return 0;
}

/* RGBA8 packing of the colour (the paper's toInt, render listing of Section 3.9).
 * Reading: per channel clamp to [0, 1], times 255, round half up, alpha 255,
 * little-endian 0xAABBGGRR.  The quantisation decision is taken in FP32, the
 * precision of the device path. */
ORC_API void orc_to_rgba8(int n, const double *rgb, uint32_t *out)
{
    for (int i = 0; i < n; ++i) {
        uint32_t px = 0xff000000u;
        for (int c = 0; c < 3; ++c) {
            float v = (float)rgb[3 * i + c];
            v = v < 0.0f ? 0.0f : (v > 1.0f ? 1.0f : v);
            uint32_t q = (uint32_t)floorf(v * 255.0f + 0.5f);
            px |= q << (8 * c);
        }
        out[i] = px;
    }
}

/* Pieces exposed for the pin tests. */
ORC_API void orc_ndc(int W, int H, double x, double y, double *uv) { ndc(W, H, x, y, uv, uv + 1); }
ORC_API double orc_camera_distance(double fov_deg) { return camera_distance(fov_deg * M_PI / 180.0); }
ORC_API int orc_primary_ray(const orc_in *in, double x, double y, double du, double dv, double *od)
{
    Ctx cx;
    int st = build_ctx(in, &cx);
    if (st) return st;
    v3 o, d;
    primary_ray(&cx, x, y, du, dv, &o, &d);
    od[0] = o.x; od[1] = o.y; od[2] = o.z; od[3] = d.x; od[4] = d.y; od[5] = d.z;
    free(cx.prim);
    free(cx.light);
    return 0;
}
ORC_API int orc_sphere_root(const double *o, const double *d, const double *c, double r, double *t)
{
    return sphere_root(V(o[0], o[1], o[2]), V(d[0], d[1], d[2]), V(c[0], c[1], c[2]), r, t);
}
ORC_API void orc_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    philox4x32_10(ctr, key, out);
}
/* Closest hit of one ray (id, t; id = -1 on a miss) and the any-hit test of one
 * shadow segment, for the brute-force and margin pin tests.  `origin` is the
 * primitive the ray leaves (-1: none); margin (nullable) receives the ray's margin. */
ORC_API int orc_closest(const orc_in *in, const double *o, const double *d, int origin, double *t,
                        double *margin)
{
    Ctx cx;
    int st = build_ctx(in, &cx);
    if (st) return -100 + st;
    Path P;
    memset(&P, 0, sizeof(P));
    P.cx = &cx;
    P.origin = origin;
    P.want_margin = margin != NULL;
    P.margin = INFINITY;
    int id = closest_hit(&P, V(o[0], o[1], o[2]), V(d[0], d[1], d[2]), t);
    if (margin) *margin = P.margin;
    free(cx.prim);
    free(cx.light);
    return id;
}
ORC_API int orc_occluded(const orc_in *in, const double *o, const double *d, double dist, int origin,
                         double *margin)
{
    Ctx cx;
    int st = build_ctx(in, &cx);
    if (st) return -100 + st;
    Path P;
    memset(&P, 0, sizeof(P));
    P.cx = &cx;
    P.origin = origin;
    P.want_margin = margin != NULL;
    P.margin = INFINITY;
    int hit = occluded(&P, V(o[0], o[1], o[2]), V(d[0], d[1], d[2]), dist);
    if (margin) *margin = P.margin;
    free(cx.prim);
    free(cx.light);
    return hit;
}

/* The path of pixel (x, y) for the pin tests: per bounce k = 0..D one record of 14
 * doubles (id, t, origin xyz, direction xyz, hit point xyz, normal xyz; id = -1 on
 * a miss, which ends the path), following the forward form's ray sequence
 * (Section 3.7.1: reflected direction d - 2 (d.n) n, origin p + eps n).  Returns
 * the number of records written. */
ORC_API int orc_trace_path(const orc_in *in, int x, int y, double *rec)
{
    Ctx cx;
    int st = build_ctx(in, &cx);
    if (st) return -100 + st;
    Path P;
    memset(&P, 0, sizeof(P));
    P.cx = &cx;
    P.origin = -1;
    v3 o, d;
    primary_ray(&cx, x, y, 0.0, 0.0, &o, &d);
    int n_rec = 0;
    for (int k = 0; k <= cx.D; ++k) {
        double t;
        const int id = closest_hit(&P, o, d, &t);
        double *r = rec + 14 * n_rec++;
        v3 p = V(0.0, 0.0, 0.0), nn = V(0.0, 0.0, 0.0);
        if (id >= 0) hit_geometry(&cx, id, o, d, t, &p, &nn);
        const double vals[14] = {id, id >= 0 ? t : 0.0, o.x, o.y, o.z, d.x, d.y, d.z, p.x, p.y, p.z, nn.x, nn.y, nn.z};
        memcpy(r, vals, sizeof(vals));
        if (id < 0) break;
        P.origin = id;
        d = sub(d, scl(nn, 2.0 * dot(d, nn)));
        o = add(p, scl(nn, cx.eps));
    }
    free(cx.prim);
    free(cx.light);
    return n_rec;
}

/* Sample points of sampled light l seen from point p at pixel (x, y), bounce k
 * (n * 3 doubles); returns n. */
ORC_API int orc_light_samples(const orc_in *in, int l, int x, int y, int k, const double *p, double *out)
{
    Ctx cx;
    int st = build_ctx(in, &cx);
    if (st) return -100 + st;
    v3 pts[ORC_MAX_SAMPLES];
    int n = 0;
    if (l >= 0 && l < cx.nl) {
        uint32_t pix = (uint32_t)y * (uint32_t)cx.W + (uint32_t)x;
        if (cx.light[l].area > 0.0) n = area_samples(&cx, pix, k, l, pts, NULL);
        else if (cx.light[l].srad > 0.0) n = vogel_samples(&cx, l, V(p[0], p[1], p[2]), pts);
    }
    for (int i = 0; i < n; ++i) { out[3 * i] = pts[i].x; out[3 * i + 1] = pts[i].y; out[3 * i + 2] = pts[i].z; }
    free(cx.prim);
    free(cx.light);
    return n;
}

/* The sky colour of one direction (Section 3.8 reading above). */
ORC_API int orc_sky(const float *tex, int w, int h, const double *d, double *rgb)
{
    if (!tex || w <= 0 || h <= 0) return -1;
    sky_lookup(tex, w, h, V(d[0], d[1], d[2]), rgb);
    return 0;
}

/* ----------------------------------------------------------- Section 3.8 physics */
/* The physics system moves the bodies by Verlet integration (Section 3.8; the
 * bodies' positions are streamed in every frame, Section 3.9).  Reading: position
 * Verlet, x_{n+1} = x_n + (x_n - x_{n-1}) + a dt^2 with a = (0, -g, 0), from the
 * current and the previous positions; contact with the ground plane n.x + pd = 0
 * (plane NULL: none): a sphere that crosses it is moved back along n until it
 * touches it, and the step's velocity v = x_{n+1} - x_n (taken before the move)
 * loses its normal component into the plane if that is at most two steps of
 * gravity (2 g dt^2: resting contact, whose component is one step of gravity; the
 * factor keeps rounding from classifying rest as an impact), else has it reversed
 * and scaled by the restitution e;
 * the previous position is set to x_{n+1} - v so that the next step continues with
 * that velocity.  pos and prev are [n][3], updated in place over `steps` steps. */
ORC_API int orc_verlet(int n, double *pos, double *prev, const double *radius, const double *plane, double dt,
                       double g, double e, int steps)
{
    if (n < 0 || steps < 0 || (n && (!pos || !prev || !radius))) return -1;
    const double gdt2 = g * dt * dt;
    for (int s = 0; s < steps; ++s) {
        for (int i = 0; i < n; ++i) {
            const v3 x = V(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]);
            const v3 xp = V(prev[3 * i], prev[3 * i + 1], prev[3 * i + 2]);
            v3 xn = add(add(x, sub(x, xp)), V(0.0, -gdt2, 0.0));
            v3 xq = x;
            if (plane) {
                const v3 nn = V(plane[0], plane[1], plane[2]);
                const double sd = dot(nn, xn) + plane[3] - radius[i];
                if (sd < 0.0) {
                    v3 v = sub(xn, x);
                    xn = sub(xn, scl(nn, sd));
                    const double vn = dot(v, nn);
                    if (vn < 0.0) v = sub(v, scl(nn, -vn <= 2.0 * gdt2 ? vn : (1.0 + e) * vn));
                    xq = sub(xn, v);
                }
            }
            pos[3 * i] = xn.x; pos[3 * i + 1] = xn.y; pos[3 * i + 2] = xn.z;
            prev[3 * i] = xq.x; prev[3 * i + 1] = xq.y; prev[3 * i + 2] = xq.z;
        }
    }
    return 0;
}
