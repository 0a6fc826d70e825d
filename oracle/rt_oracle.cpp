// Plain FP64 CPU oracle of the differentiable radio ray tracer.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference
// against which the CUDA library is checked.  Only the tests, the smoke check and
// the CPU-baseline leg of the benchmark load it; the product path never does.  It
// shares no code, header, table or helper with the CUDA library.
//
// Every step follows the paper "Learning Radio Environments by Differentiable Ray
// Tracing" (Hoydis et al., arXiv 2311.18558) in its own order and notation:
//   * path tracing: candidate primitives by shooting-and-bouncing rays, then exact
//     specular chains by the image method (Sec. II-F);
//   * transfer function of a path: basis changes D_j (Eq. rel1 / basis_transform),
//     scattering maps F_j (Eq. rel2, Eq. init, Eq. specular_reflection), Fresnel
//     coefficients (Eq. fresnel-1/2), complex permittivity eta (Sec. II-D);
//   * path coefficient a_i and delay tau_i (Eq. cfr_cont, Eq. transfer_function);
//   * CFR H[n] = H(f + n df), n = -N/2 .. N/2-1 (Sec. II-A).
// Readings where the paper is silent (spreading factor, reflection basis vectors,
// Fibonacci launch, hit rules, duplicate rule) are stated where they are used.
//
// Nothing here is blocked, fused or reordered for speed beyond one OpenMP loop
// over independent rays or receivers.

#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <vector>

typedef std::complex<double> cplx;

static const double kC0 = 299792458.0;          // speed of light [m/s] (CODATA)
static const double kEps0 = 8.8541878128e-12;   // vacuum permittivity [F/m] (CODATA)
static const double kPi = 3.14159265358979323846;

struct Vec3 {
    double x, y, z;
};
static inline Vec3 v3(double x, double y, double z) { return Vec3{x, y, z}; }
static inline Vec3 operator+(Vec3 a, Vec3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
static inline Vec3 operator-(Vec3 a, Vec3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
static inline Vec3 operator*(double s, Vec3 a) { return v3(s * a.x, s * a.y, s * a.z); }
static inline double dot(Vec3 a, Vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static inline Vec3 cross(Vec3 a, Vec3 b) {
    return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static inline double norm(Vec3 a) { return std::sqrt(dot(a, a)); }
static inline Vec3 unit(Vec3 a) { return (1.0 / norm(a)) * a; }
static inline double comp(Vec3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

// ---------------------------------------------------------------------------
// Scene: triangles, their planes, and a median-split BVH used only to speed up
// the closest-hit and any-hit queries.  The BVH never changes a result: every
// query is also available by brute force over all triangles, and the tests check
// that both give the identical answer.

struct Box {
    Vec3 lo, hi;
};

struct Node {
    Box box;
    int left, right;   // children, -1 for a leaf
    int first, count;  // leaf range in `order`
};

struct Scene {
    int T;
    std::vector<Vec3> a, b, c;   // triangle vertices
    std::vector<Vec3> n;         // unit geometric normal (b-a)x(c-a)
    double diag;                 // diagonal of the scene's bounding box
    std::vector<Node> nodes;
    std::vector<int> order;
};

static Box tri_box(const Scene& s, int t) {
    Box bx;
    bx.lo = v3(std::min({s.a[t].x, s.b[t].x, s.c[t].x}), std::min({s.a[t].y, s.b[t].y, s.c[t].y}),
               std::min({s.a[t].z, s.b[t].z, s.c[t].z}));
    bx.hi = v3(std::max({s.a[t].x, s.b[t].x, s.c[t].x}), std::max({s.a[t].y, s.b[t].y, s.c[t].y}),
               std::max({s.a[t].z, s.b[t].z, s.c[t].z}));
    return bx;
}

static int build_node(Scene& s, int first, int count) {
    Node nd;
    nd.box = tri_box(s, s.order[first]);
    for (int i = first + 1; i < first + count; ++i) {
        Box b = tri_box(s, s.order[i]);
        nd.box.lo = v3(std::min(nd.box.lo.x, b.lo.x), std::min(nd.box.lo.y, b.lo.y), std::min(nd.box.lo.z, b.lo.z));
        nd.box.hi = v3(std::max(nd.box.hi.x, b.hi.x), std::max(nd.box.hi.y, b.hi.y), std::max(nd.box.hi.z, b.hi.z));
    }
    // Pad the box so that rounding in the slab test can never prune a triangle
    // lying on the box boundary.
    double pad = 1e-9 * s.diag;
    nd.box.lo = nd.box.lo - v3(pad, pad, pad);
    nd.box.hi = nd.box.hi + v3(pad, pad, pad);
    nd.left = nd.right = -1;
    nd.first = first;
    nd.count = count;
    int id = (int)s.nodes.size();
    s.nodes.push_back(nd);
    if (count <= 4) return id;
    Vec3 ext = nd.box.hi - nd.box.lo;
    int axis = (ext.x >= ext.y && ext.x >= ext.z) ? 0 : (ext.y >= ext.z ? 1 : 2);
    std::vector<int>::iterator beg = s.order.begin() + first;
    std::sort(beg, beg + count, [&](int p, int q) {
        double cp = comp(s.a[p] + s.b[p] + s.c[p], axis), cq = comp(s.a[q] + s.b[q] + s.c[q], axis);
        return cp < cq || (cp == cq && p < q);
    });
    int half = count / 2;
    int l = build_node(s, first, half);
    int r = build_node(s, first + half, count - half);
    s.nodes[id].left = l;
    s.nodes[id].right = r;
    return id;
}

// Slab test: does the ray o + t d, t in [tmin, tmax], touch the box?
static bool box_hit(const Box& bx, Vec3 o, Vec3 d, double tmin, double tmax) {
    double t0 = tmin, t1 = tmax;
    for (int k = 0; k < 3; ++k) {
        double ok = comp(o, k), dk = comp(d, k), lo = comp(bx.lo, k), hi = comp(bx.hi, k);
        if (dk == 0.0) {
            if (ok < lo || ok > hi) return false;
            continue;
        }
        double ta = (lo - ok) / dk, tb = (hi - ok) / dk;
        if (ta > tb) std::swap(ta, tb);
        t0 = std::max(t0, ta);
        t1 = std::min(t1, tb);
        if (t0 > t1) return false;
    }
    return true;
}

// Degenerate geometry (the paper is silent on it).  Reading: a triangle counts
// as closed and grown by kTol relative to its size, so a point or ray exactly on
// an edge shared by two triangles belongs to both, whatever the rounding; the
// duplicate rule and the tie rule below then pick one of them.
static const double kTol = 1e-9;      // relative growth of every triangle
static const double kTieTol = 1e-12;  // relative t-difference treated as a tie

// Watertight ray/triangle intersection (Woop, Benthin and Wald, "Watertight
// Ray/Triangle Intersection", JCGT 2013), evaluated in FP64, with the scaled
// barycentrics U, V, W allowed down to -kTol (|U| + |V| + |W|).  A ray lying in
// the triangle's plane misses.  Returns the ray parameter t or -1 for a miss.
static double tri_hit(const Scene& s, int t, Vec3 o, Vec3 d) {
    double dd[3] = {d.x, d.y, d.z};
    int kz = 0;
    if (std::fabs(dd[1]) > std::fabs(dd[kz])) kz = 1;
    if (std::fabs(dd[2]) > std::fabs(dd[kz])) kz = 2;
    int kx = (kz + 1) % 3, ky = (kx + 1) % 3;
    if (dd[kz] < 0.0) std::swap(kx, ky);
    double Sx = dd[kx] / dd[kz], Sy = dd[ky] / dd[kz], Sz = 1.0 / dd[kz];
    Vec3 A = s.a[t] - o, B = s.b[t] - o, C = s.c[t] - o;
    double Ax = comp(A, kx) - Sx * comp(A, kz), Ay = comp(A, ky) - Sy * comp(A, kz);
    double Bx = comp(B, kx) - Sx * comp(B, kz), By = comp(B, ky) - Sy * comp(B, kz);
    double Cx = comp(C, kx) - Sx * comp(C, kz), Cy = comp(C, ky) - Sy * comp(C, kz);
    double U = Cx * By - Cy * Bx;
    double V = Ax * Cy - Ay * Cx;
    double W = Bx * Ay - By * Ax;
    double m = kTol * (std::fabs(U) + std::fabs(V) + std::fabs(W));
    if ((U < -m || V < -m || W < -m) && (U > m || V > m || W > m)) return -1.0;
    double det = U + V + W;
    if (!(std::fabs(det) > 3.0 * m)) return -1.0;
    double Az = Sz * comp(A, kz), Bz = Sz * comp(B, kz), Cz = Sz * comp(C, kz);
    double T = U * Az + V * Bz + W * Cz;
    return T / det;
}

// All hits with tmin < t <= tmax (skipping `skip`): calls f(t, triangle).
template <typename F>
static void each_hit(const Scene& s, Vec3 o, Vec3 d, double tmin, double tmax, int skip, bool use_bvh, F f) {
    if (!use_bvh) {
        for (int t = 0; t < s.T; ++t) {
            if (t == skip) continue;
            double th = tri_hit(s, t, o, d);
            if (th > tmin && th <= tmax) f(th, t);
        }
        return;
    }
    std::vector<int> stack;
    stack.push_back(0);
    while (!stack.empty()) {
        int ni = stack.back();
        stack.pop_back();
        const Node& nd = s.nodes[ni];
        if (!box_hit(nd.box, o, d, tmin, tmax)) continue;
        if (nd.left < 0) {
            for (int i = nd.first; i < nd.first + nd.count; ++i) {
                int t = s.order[i];
                if (t == skip) continue;
                double th = tri_hit(s, t, o, d);
                if (th > tmin && th <= tmax) f(th, t);
            }
        } else {
            stack.push_back(nd.left);
            stack.push_back(nd.right);
        }
    }
}

// Closest hit with t > tmin, skipping triangle `skip`: the smallest t over all
// hits, then, among the hits with t within kTieTol (relative) of it, the lowest
// triangle index -- an answer that does not depend on the visiting order.
static int closest_hit(const Scene& s, Vec3 o, Vec3 d, double tmin, int skip, bool use_bvh, double* t_out) {
    double bt = INFINITY;
    each_hit(s, o, d, tmin, INFINITY, skip, use_bvh, [&](double th, int) { bt = std::min(bt, th); });
    *t_out = bt;
    if (!(bt < INFINITY)) return -1;
    int best = -1;
    each_hit(s, o, d, tmin, bt + kTieTol * bt, skip, use_bvh, [&](double, int t) {
        if (best < 0 || t < best) best = t;
    });
    return best;
}

// Any hit with tmin < t < tmax, skipping triangles skip0 and skip1.
static bool any_hit(const Scene& s, Vec3 o, Vec3 d, double tmin, double tmax, int skip0, int skip1) {
    std::vector<int> stack;
    stack.push_back(0);
    while (!stack.empty()) {
        int ni = stack.back();
        stack.pop_back();
        const Node& nd = s.nodes[ni];
        if (!box_hit(nd.box, o, d, tmin, tmax)) continue;
        if (nd.left < 0) {
            for (int i = nd.first; i < nd.first + nd.count; ++i) {
                int t = s.order[i];
                if (t == skip0 || t == skip1) continue;
                double th = tri_hit(s, t, o, d);
                if (th > tmin && th < tmax) return true;
            }
        } else {
            stack.push_back(nd.left);
            stack.push_back(nd.right);
        }
    }
    return false;
}

// Point-in-triangle test for a point on (or numerically next to) the triangle's
// plane: the three edge functions along the normal, divided by |n|^2 (i.e. the
// barycentric coordinates), are >= -kTol (closed triangle grown by kTol).
static bool point_in_tri(const Scene& s, int t, Vec3 p) {
    Vec3 nn = cross(s.b[t] - s.a[t], s.c[t] - s.a[t]);
    double n2 = dot(nn, nn);
    double e0 = dot(nn, cross(s.b[t] - s.a[t], p - s.a[t])) / n2;
    double e1 = dot(nn, cross(s.c[t] - s.b[t], p - s.b[t])) / n2;
    double e2 = dot(nn, cross(s.a[t] - s.c[t], p - s.c[t])) / n2;
    return e0 >= -kTol && e1 >= -kTol && e2 >= -kTol;
}

static bool coplanar(const Scene& s, int t, int u) {
    if (t == u) return true;
    Vec3 cr = cross(s.n[t], s.n[u]);
    if (norm(cr) > 1e-9) return false;
    double dt = dot(s.n[t], s.a[t]);
    double du = dot(s.n[t], s.a[u]);
    return std::fabs(dt - du) <= 1e-9 * s.diag;
}

// ---------------------------------------------------------------------------
// Fibonacci-sphere launch directions.  The paper does not print its launch
// pattern.  Reading: the Fibonacci lattice on the sphere (Gonzalez 2010),
//   z_i = 1 - (2i+1)/N,  r_i = sqrt(1 - z_i^2),  phi_i = 2 pi frac(i g),  g = (sqrt5 - 1)/2,
// with frac(i g) taken from the 32-bit golden-ratio Weyl sequence
// (i * 0x9E3779B9 mod 2^32) / 2^32, and sin, cos of phi from the Taylor series
// of sin (to theta^11) and cos (to theta^12) on the octant theta in [0, pi/4]
// plus the octant symmetries.  z is one IEEE FP64 division and subtraction
// rounded to FP32; every other step is one IEEE FP32 operation (no contraction),
// so the canonical FP32 ray set is reproduced bit for bit by any IEEE
// implementation.  The oracle traces these FP32 directions in FP64.
static void sincos_turn(uint32_t k, float* s_out, float* c_out) {
    uint32_t oct = k >> 29;                                           // octant of the turn
    float y = (float)(k & 0x1fffffffu) * (1.0f / 536870912.0f);      // position in it, [0, 1)
    float t = (oct & 1u) ? 1.0f - y : y;                              // distance to the nearest multiple of pi/2
    float th = t * 0.785398185253143310546875f;                       // times pi/4 (FP32)
    float x = th * th;
    float ps = -2.50521083854417187751e-08f;                          // -1/11!
    ps = ps * x + 2.75573192239858906526e-06f;                        // 1/9!
    ps = ps * x + -1.98412698412698412698e-04f;                       // -1/7!
    ps = ps * x + 8.33333333333333333333e-03f;                        // 1/5!
    ps = ps * x + -1.66666666666666666667e-01f;                       // -1/3!
    ps = ps * x + 1.0f;
    float sn = ps * th;                                               // sin(theta)
    float pc = 2.08767569878680989792e-09f;                           // 1/12!
    pc = pc * x + -2.75573192239858906526e-07f;                       // -1/10!
    pc = pc * x + 2.48015873015873015873e-05f;                        // 1/8!
    pc = pc * x + -1.38888888888888888889e-03f;                       // -1/6!
    pc = pc * x + 4.16666666666666666667e-02f;                        // 1/4!
    pc = pc * x + -0.5f;                                              // -1/2!
    pc = pc * x + 1.0f;                                               // cos(theta)
    // angle = quadrant * pi/2 + sign * theta
    uint32_t quadrant = ((oct + 1u) >> 1) & 3u;
    float ss = (oct & 1u) ? -sn : sn;
    float cs = pc;
    switch (quadrant) {
        case 0: *s_out = ss; *c_out = cs; break;
        case 1: *s_out = cs; *c_out = -ss; break;
        case 2: *s_out = -ss; *c_out = -cs; break;
        default: *s_out = -cs; *c_out = ss; break;
    }
}

static void fibonacci_dir(int64_t i, int64_t N, float out[3]) {
    float z = (float)(1.0 - (double)(2 * i + 1) / (double)N);
    float r = std::sqrt(1.0f - z * z);
    float s, c;
    sincos_turn((uint32_t)((uint64_t)i * 0x9E3779B9ull), &s, &c);
    out[0] = r * c;
    out[1] = r * s;
    out[2] = z;
}

// One SBR ray: up to D specular bounces (reflected direction k_r = k_i - 2(k_i.n)n,
// Sec. II-D), each leaving triangle excluded from the next closest-hit query.
// Writes the triangle sequence (-1 after the ray escapes) and returns #hits.
static int sbr_ray(const Scene& s, Vec3 tx, Vec3 dir, int D, double tmin, bool use_bvh, int* seq) {
    Vec3 o = tx, d = dir;
    int prev = -1, hits = 0;
    for (int b = 0; b < D; ++b) seq[b] = -1;
    for (int b = 0; b < D; ++b) {
        double th;
        int t = closest_hit(s, o, d, tmin, prev, use_bvh, &th);
        if (t < 0) break;
        seq[b] = t;
        hits++;
        Vec3 p = o + th * d;
        Vec3 nn = s.n[t];
        d = d - (2.0 * dot(d, nn)) * nn;
        o = p;
        prev = t;
    }
    return hits;
}

// ---------------------------------------------------------------------------
// Image method (Sec. II-F): for a candidate sequence (t_1..t_q) and a receiver,
// mirror the transmitter successively in the planes of t_1..t_q, then trace back
// from the receiver towards the images; each back-traced segment must cross the
// plane strictly between its end points (0 < u < 1) and the crossing must lie in
// the closed triangle.  Then every segment s_j -> s_{j+1} must be free of other
// triangles for t in (eps, len - eps), the end triangles excluded.
// Returns true and fills pts (q+2 points: Tx, s_1..s_q, Rx) if the path is valid.
static bool image_path(const Scene& s, Vec3 tx, Vec3 rx, const int* seq, int q, double eps, Vec3* pts,
                       bool* on_edge) {
    std::vector<Vec3> img(q + 1);
    img[0] = tx;
    for (int j = 1; j <= q; ++j) {
        int t = seq[j - 1];
        Vec3 nn = s.n[t];
        img[j] = img[j - 1] - (2.0 * dot(img[j - 1] - s.a[t], nn)) * nn;
    }
    pts[0] = tx;
    pts[q + 1] = rx;
    for (int j = q; j >= 1; --j) {
        int t = seq[j - 1];
        Vec3 nn = s.n[t];
        Vec3 from = pts[j + 1];
        Vec3 dir = img[j] - from;
        double den = dot(nn, dir);
        if (den == 0.0) return false;
        double u = dot(nn, s.a[t] - from) / den;
        if (!(u > 0.0 && u < 1.0)) return false;
        Vec3 p = from + u * dir;
        if (!point_in_tri(s, t, p)) return false;
        pts[j] = p;
    }
    *on_edge = false;
    for (int j = 0; j <= q; ++j) {
        Vec3 d = pts[j + 1] - pts[j];
        double len = norm(d);
        if (len <= eps) return false;
        int s0 = j >= 1 ? seq[j - 1] : -1;
        int s1 = j + 1 <= q ? seq[j] : -1;
        if (any_hit(s, pts[j], d, eps / len, 1.0 - eps / len, s0, s1)) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Antenna basis vectors theta_hat, phi_hat of direction k (notation of Sec. I).
// The azimuth of a vertical direction is undefined; reading: phi = 0 there.
static void sph_basis(Vec3 k, Vec3* th, Vec3* ph) {
    double theta = std::acos(std::max(-1.0, std::min(1.0, k.z)));
    double phi = (k.x == 0.0 && k.y == 0.0) ? 0.0 : std::atan2(k.y, k.x);
    *th = v3(std::cos(theta) * std::cos(phi), std::cos(theta) * std::sin(phi), -std::sin(theta));
    *ph = v3(-std::sin(phi), std::cos(phi), 0.0);
}

// Complex relative permittivity eta = eps_r - j sigma / (eps0 omega) (Sec. II-D).
static cplx permittivity(double eps_r, double sigma, double freq) {
    return cplx(eps_r, -sigma / (kEps0 * 2.0 * kPi * freq));
}

// Fresnel reflection coefficients (Eq. fresnel-1, fresnel-2) with the principal
// complex square root.
static void fresnel(cplx eta, double cos_i, cplx* r_perp, cplx* r_par) {
    double sin2 = 1.0 - cos_i * cos_i;
    cplx s = std::sqrt(eta - sin2);
    *r_perp = (cos_i - s) / (cos_i + s);
    *r_par = (eta * cos_i - s) / (eta * cos_i + s);
}

// d r_perp / d eta and d r_par / d eta (derivatives of Eq. fresnel-1/2).
static void fresnel_deta(cplx eta, double cos_i, cplx* d_perp, cplx* d_par) {
    double sin2 = 1.0 - cos_i * cos_i;
    cplx s = std::sqrt(eta - sin2);
    *d_perp = -cos_i / (s * (cos_i + s) * (cos_i + s));
    *d_par = cos_i * (eta - 2.0 * sin2) / (s * (eta * cos_i + s) * (eta * cos_i + s));
}

struct PathMaterials {
    const int32_t* tri_material;
    const float* eps_r;
    const float* sigma;
    const uint8_t* is_pec;
    int per_triangle;
};

// Transfer chain of one specular path (Sec. II-C, II-D):
//   E_0 = C_T;  F_0(E) = e^{-j 2 pi d_1 / lambda} / d_1 E;
//   for each bounce j: E <- D_j E (basis change), then
//                      E <- diag(R r_perp, R r_par) E A_j e^{-j 2 pi d_{j+1} / lambda};
//   E_{Q+1} = D_{Q+1} E = T(C_T) e^{-j 2 pi f tau},  a = lambda/(4 pi) C_R^H T(C_T).
// Spreading factor (the paper cites it without printing it): for planar facets the
// reflected wave front stays spherical about the image source, so
// A_j = rho_j / (rho_j + d_{j+1}) with rho_j = d_1 + ... + d_j.  S = 0 (R = 1).
// Polarisation model Eq. polarization_model with zeta = 0 (vertical) at both ends.
// Reflection basis (McNamara Eq. 3.3-3.8, cited, not printed): e_perp = k_i x n / |k_i x n|,
// e_par_in = e_perp x k_i, e_par_out = e_perp x k_r, n facing the incident wave.
//
// Outputs: a, and when `grad` is non-null, d a / d eta_j for every bounce.
struct ChainOut {
    cplx a;
    cplx da_deta[8];
    int mat[8];
    bool pec[8];
};

static void path_chain(const Scene& s, const PathMaterials& m, const Vec3* pts, const int* seq, int q,
                       double freq, double gain_tx, double gain_rx, int ni_mode, ChainOut* out) {
    const double lam = kC0 / freq;
    std::vector<double> d(q + 2);
    std::vector<Vec3> k(q + 2);
    double L = 0.0;
    for (int j = 1; j <= q + 1; ++j) {
        Vec3 dv = pts[j] - pts[j - 1];
        d[j] = norm(dv);
        k[j] = (1.0 / d[j]) * dv;
        L += d[j];
    }
    const double tau = L / kC0;  // tau = (lambda f)^-1 sum d_q

    // out_0 basis: the transmit antenna's theta_hat / phi_hat along the AoD k_1.
    Vec3 out_p, out_q;
    sph_basis(k[1], &out_p, &out_q);
    cplx E[2] = {std::sqrt(gain_tx) * 1.0, std::sqrt(gain_tx) * 0.0};  // C_T, zeta = 0

    // F_0
    cplx ph1 = std::polar(1.0, -2.0 * kPi * d[1] / lam);
    E[0] *= ph1 / d[1];
    E[1] *= ph1 / d[1];

    // Stored for the adjoint: incoming field after the basis change of bounce j,
    // and the reflection matrix of bounce j.
    std::vector<cplx> vin0(q + 1), vin1(q + 1), rp(q + 1), rl(q + 1);
    std::vector<double> Dm(4 * (q + 2));
    std::vector<double> spread(q + 1);
    std::vector<cplx> phase(q + 1);

    double rho = d[1];
    for (int j = 1; j <= q; ++j) {
        int t = seq[j - 1];
        Vec3 nn = s.n[t];
        if (dot(k[j], nn) > 0.0) nn = -1.0 * nn;   // normal facing the incident wave
        double cos_i = -dot(k[j], nn);
        Vec3 kr = k[j + 1];
        Vec3 cr = cross(k[j], nn);
        Vec3 e_perp;
        if (norm(cr) > 1e-12) {
            e_perp = unit(cr);
        } else {
            // Normal incidence: any unit vector transverse to k_i serves; take the
            // previous outgoing p-vector (mode 0) or the world x axis (mode 1),
            // made orthogonal to k_i.
            Vec3 ref = ni_mode == 0 ? out_p : v3(1.0, 0.0, 0.0);
            if (ni_mode != 0 && norm(cross(ref, k[j])) < 1e-6) ref = v3(0.0, 1.0, 0.0);
            e_perp = unit(ref - dot(ref, k[j]) * k[j]);
        }
        Vec3 in_p = e_perp, in_q = cross(e_perp, k[j]);
        // D_j (Eq. basis_transform)
        double D00 = dot(in_p, out_p), D01 = dot(in_p, out_q);
        double D10 = dot(in_q, out_p), D11 = dot(in_q, out_q);
        Dm[4 * j + 0] = D00; Dm[4 * j + 1] = D01; Dm[4 * j + 2] = D10; Dm[4 * j + 3] = D11;
        cplx e0 = D00 * E[0] + D01 * E[1];
        cplx e1 = D10 * E[0] + D11 * E[1];
        vin0[j] = e0;
        vin1[j] = e1;
        // F_j (Eq. specular_reflection)
        int mi = m.per_triangle ? t : m.tri_material[t];
        bool pec = m.is_pec[mi] != 0;
        cplx r_perp, r_par;
        if (pec) {
            r_perp = -1.0;   // limit of Eq. fresnel-1/2 as |eta| -> infinity
            r_par = 1.0;
        } else {
            fresnel(permittivity(m.eps_r[mi], m.sigma[mi], freq), cos_i, &r_perp, &r_par);
        }
        rp[j] = r_perp;
        rl[j] = r_par;
        out->mat[j - 1] = mi;
        out->pec[j - 1] = pec;
        double A = rho / (rho + d[j + 1]);
        spread[j] = A;
        phase[j] = std::polar(1.0, -2.0 * kPi * d[j + 1] / lam);
        E[0] = r_perp * e0 * A * phase[j];
        E[1] = r_par * e1 * A * phase[j];
        rho += d[j + 1];
        out_p = e_perp;
        out_q = cross(e_perp, kr);
    }
    // D_{Q+1}: into the receive antenna's basis along the AoA direction -k_{Q+1}.
    Vec3 rx_p, rx_q;
    sph_basis(-1.0 * k[q + 1], &rx_p, &rx_q);
    double D00 = dot(rx_p, out_p), D01 = dot(rx_p, out_q);
    double D10 = dot(rx_q, out_p), D11 = dot(rx_q, out_q);
    Dm[4 * (q + 1) + 0] = D00; Dm[4 * (q + 1) + 1] = D01; Dm[4 * (q + 1) + 2] = D10; Dm[4 * (q + 1) + 3] = D11;
    cplx Ef0 = D00 * E[0] + D01 * E[1];
    cplx Ef1 = D10 * E[0] + D11 * E[1];
    (void)Ef1;
    // Factor out exp(-j 2 pi f tau) and project on C_R = sqrt(g_R) [1, 0].
    cplx unphase = std::polar(1.0, 2.0 * kPi * freq * tau);
    cplx a = lam / (4.0 * kPi) * std::sqrt(gain_rx) * Ef0 * unphase;
    out->a = a;

    // Adjoint: a = K * l_j . diag(r_perp_j, r_par_j) . v_j, with the row vector
    // l_j = C_R^T D_{Q+1} Gamma_Q D_Q ... D_{j+1} (times the scalar factors after
    // bounce j) and v_j the field after D_j.  Walk j = Q..1 keeping l_j.
    cplx l0 = lam / (4.0 * kPi) * std::sqrt(gain_rx) * unphase * Dm[4 * (q + 1) + 0];
    cplx l1 = lam / (4.0 * kPi) * std::sqrt(gain_rx) * unphase * Dm[4 * (q + 1) + 1];
    for (int j = q; j >= 1; --j) {
        cplx fac = spread[j] * phase[j];
        cplx da_drp = l0 * fac * vin0[j];
        cplx da_drl = l1 * fac * vin1[j];
        if (out->pec[j - 1]) {
            out->da_deta[j - 1] = 0.0;
        } else {
            int mi = out->mat[j - 1];
            Vec3 nn = s.n[seq[j - 1]];
            if (dot(k[j], nn) > 0.0) nn = -1.0 * nn;
            double cos_i = -dot(k[j], nn);
            cplx dp, dl;
            fresnel_deta(permittivity(m.eps_r[mi], m.sigma[mi], freq), cos_i, &dp, &dl);
            out->da_deta[j - 1] = da_drp * dp + da_drl * dl;
        }
        // l_{j-1} = l_j . Gamma_j . (fac) . D_j
        cplx g0 = l0 * rp[j] * fac, g1 = l1 * rl[j] * fac;
        l0 = g0 * Dm[4 * j + 0] + g1 * Dm[4 * j + 2];
        l1 = g0 * Dm[4 * j + 1] + g1 * Dm[4 * j + 3];
    }
}

// ---------------------------------------------------------------------------
// Path store returned to Python.

struct Paths {
    int Dmax;
    std::vector<int32_t> rx, depth, seq;  // seq: P x Dmax, -1 padded
    std::vector<double> pts;              // P x (Dmax+2) x 3
    std::vector<double> tau;
    std::vector<int32_t> ray;             // diffuse paths: the launch ray that found the path
};

static bool seq_less(const int* a, const int* b, int q) {
    for (int j = 0; j < q; ++j)
        if (a[j] != b[j]) return a[j] < b[j];
    return false;
}

extern "C" {

void* orc_scene_create(const float* verts, int n_verts, const int32_t* tris, int n_tris) {
    (void)n_verts;
    Scene* s = new Scene();
    s->T = n_tris;
    s->a.resize(n_tris);
    s->b.resize(n_tris);
    s->c.resize(n_tris);
    s->n.resize(n_tris);
    Vec3 lo = v3(INFINITY, INFINITY, INFINITY), hi = v3(-INFINITY, -INFINITY, -INFINITY);
    for (int t = 0; t < n_tris; ++t) {
        const float* p0 = verts + 3 * tris[3 * t + 0];
        const float* p1 = verts + 3 * tris[3 * t + 1];
        const float* p2 = verts + 3 * tris[3 * t + 2];
        s->a[t] = v3(p0[0], p0[1], p0[2]);
        s->b[t] = v3(p1[0], p1[1], p1[2]);
        s->c[t] = v3(p2[0], p2[1], p2[2]);
        s->n[t] = unit(cross(s->b[t] - s->a[t], s->c[t] - s->a[t]));
        for (Vec3 p : {s->a[t], s->b[t], s->c[t]}) {
            lo = v3(std::min(lo.x, p.x), std::min(lo.y, p.y), std::min(lo.z, p.z));
            hi = v3(std::max(hi.x, p.x), std::max(hi.y, p.y), std::max(hi.z, p.z));
        }
    }
    s->diag = norm(hi - lo);
    s->order.resize(n_tris);
    for (int t = 0; t < n_tris; ++t) s->order[t] = t;
    build_node(*s, 0, n_tris);
    return s;
}

void orc_scene_free(void* h) { delete (Scene*)h; }

double orc_scene_diag(void* h) { return ((Scene*)h)->diag; }

int orc_bvh_nodes(void* h) { return (int)((Scene*)h)->nodes.size(); }

// Closest hit for n rays (o, d as FP64 triples).  skip[i] < 0 skips nothing.
void orc_closest_hit(void* h, int64_t n, const double* o, const double* d, double tmin, const int32_t* skip,
                     int use_bvh, int32_t* tri_out, double* t_out) {
    const Scene& s = *(Scene*)h;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        double th;
        int t = closest_hit(s, v3(o[3 * i], o[3 * i + 1], o[3 * i + 2]), v3(d[3 * i], d[3 * i + 1], d[3 * i + 2]),
                            tmin, skip ? skip[i] : -1, use_bvh != 0, &th);
        tri_out[i] = t;
        t_out[i] = t >= 0 ? th : INFINITY;
    }
}

void orc_fibonacci(int64_t n, float* dirs) {
    for (int64_t i = 0; i < n; ++i) fibonacci_dir(i, n, dirs + 3 * i);
}

// Per-ray SBR sequences (N x D, -1 padded), for checking the launch itself.
void orc_sbr_rays(void* h, const double* tx, int64_t n_rays, int D, int use_bvh, int32_t* seqs) {
    const Scene& s = *(Scene*)h;
    double tmin = 1e-6 * s.diag;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n_rays; ++i) {
        float f[3];
        fibonacci_dir(i, n_rays, f);
        sbr_ray(s, v3(tx[0], tx[1], tx[2]), v3(f[0], f[1], f[2]), D, tmin, use_bvh != 0, seqs + (size_t)D * i);
    }
}

// Candidate set: the empty sequence (line of sight) and every non-empty prefix of
// every ray's sequence, unique, ordered by (length, lexicographic).
void* orc_candidates(void* h, const double* tx, int64_t n_rays, int D) {
    const Scene& s = *(Scene*)h;
    std::vector<int32_t> seqs((size_t)n_rays * D);
    orc_sbr_rays(h, tx, n_rays, D, 1, seqs.data());
    std::set<std::vector<int>> uniq;
    uniq.insert(std::vector<int>());
    for (int64_t i = 0; i < n_rays; ++i) {
        std::vector<int> pre;
        for (int b = 0; b < D; ++b) {
            int t = seqs[(size_t)D * i + b];
            if (t < 0) break;
            pre.push_back(t);
            uniq.insert(pre);
        }
    }
    (void)s;
    std::vector<std::vector<int>> v(uniq.begin(), uniq.end());
    std::stable_sort(v.begin(), v.end(), [](const std::vector<int>& x, const std::vector<int>& y) {
        if (x.size() != y.size()) return x.size() < y.size();
        return x < y;
    });
    std::vector<int32_t>* out = new std::vector<int32_t>();
    out->push_back(D);
    out->push_back((int32_t)v.size());
    for (auto& q : v) {
        for (int b = 0; b < D; ++b) out->push_back(b < (int)q.size() ? q[b] : -1);
    }
    return out;
}

int64_t orc_candidates_count(void* c) { return (*(std::vector<int32_t>*)c)[1]; }

void orc_candidates_get(void* c, int32_t* seqs) {
    std::vector<int32_t>& v = *(std::vector<int32_t>*)c;
    std::memcpy(seqs, v.data() + 2, sizeof(int32_t) * (v.size() - 2));
}

void orc_candidates_free(void* c) { delete (std::vector<int32_t>*)c; }

// Image method over every (candidate, receiver) pair, then the coplanar-duplicate
// rule (the paper is silent on it): two valid paths of one receiver whose
// triangles are pairwise coplanar and whose points agree within 1e-9 * diag are
// the same geometric path (a reflection point on an edge shared by coplanar
// triangles); only the lexicographically smallest triangle sequence is kept.
void* orc_image_method(void* h, const double* tx, const double* rx, int n_rx, void* cand_h) {
    const Scene& s = *(Scene*)h;
    std::vector<int32_t>& cv = *(std::vector<int32_t>*)cand_h;
    int D = cv[0];
    int64_t K = cv[1];
    const int32_t* cands = cv.data() + 2;
    double eps = 1e-6 * s.diag;
    Vec3 txv = v3(tx[0], tx[1], tx[2]);
    std::vector<Paths> per_rx(n_rx);
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < n_rx; ++r) {
        Vec3 rxv = v3(rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]);
        Paths& pr = per_rx[r];
        std::vector<Vec3> pts(D + 2);
        for (int64_t k = 0; k < K; ++k) {
            const int32_t* sq = cands + (size_t)D * k;
            int q = 0;
            while (q < D && sq[q] >= 0) q++;
            bool on_edge;
            if (!image_path(s, txv, rxv, sq, q, eps, pts.data(), &on_edge)) continue;
            pr.depth.push_back(q);
            for (int b = 0; b < D; ++b) pr.seq.push_back(b < q ? sq[b] : -1);
            for (int j = 0; j < D + 2; ++j) {
                Vec3 p = j < q + 2 ? pts[j] : v3(0, 0, 0);
                if (j == q + 1) p = rxv;
                pr.pts.push_back(p.x);
                pr.pts.push_back(p.y);
                pr.pts.push_back(p.z);
            }
        }
        // coplanar-duplicate rule
        int P = (int)pr.depth.size();
        std::vector<char> drop(P, 0);
        for (int i = 0; i < P; ++i) {
            for (int j = 0; j < P; ++j) {
                if (i == j || drop[j] || pr.depth[i] != pr.depth[j]) continue;
                int q = pr.depth[i];
                bool same = true;
                for (int b = 0; b < q && same; ++b)
                    same = coplanar(s, pr.seq[(size_t)D * i + b], pr.seq[(size_t)D * j + b]);
                for (int b = 1; b <= q && same; ++b) {
                    const double* pi = &pr.pts[((size_t)(D + 2) * i + b) * 3];
                    const double* pj = &pr.pts[((size_t)(D + 2) * j + b) * 3];
                    double dd = std::sqrt((pi[0] - pj[0]) * (pi[0] - pj[0]) + (pi[1] - pj[1]) * (pi[1] - pj[1]) +
                                          (pi[2] - pj[2]) * (pi[2] - pj[2]));
                    same = dd <= 1e-9 * s.diag;
                }
                if (same && seq_less(&pr.seq[(size_t)D * j], &pr.seq[(size_t)D * i], q)) {
                    drop[i] = 1;
                    break;
                }
            }
        }
        Paths kept;
        for (int i = 0; i < P; ++i) {
            if (drop[i]) continue;
            kept.depth.push_back(pr.depth[i]);
            for (int b = 0; b < D; ++b) kept.seq.push_back(pr.seq[(size_t)D * i + b]);
            double L = 0.0;
            int q = pr.depth[i];
            for (int j = 0; j < D + 2; ++j)
                for (int c = 0; c < 3; ++c) kept.pts.push_back(pr.pts[((size_t)(D + 2) * i + j) * 3 + c]);
            for (int j = 1; j <= q + 1; ++j) {
                const double* p0 = &pr.pts[((size_t)(D + 2) * i + j - 1) * 3];
                const double* p1 = &pr.pts[((size_t)(D + 2) * i + j) * 3];
                L += std::sqrt((p1[0] - p0[0]) * (p1[0] - p0[0]) + (p1[1] - p0[1]) * (p1[1] - p0[1]) +
                               (p1[2] - p0[2]) * (p1[2] - p0[2]));
            }
            kept.tau.push_back(L / kC0);
        }
        pr = kept;
    }
    Paths* all = new Paths();
    all->Dmax = D;
    for (int r = 0; r < n_rx; ++r) {
        Paths& pr = per_rx[r];
        for (size_t i = 0; i < pr.depth.size(); ++i) all->rx.push_back(r);
        all->depth.insert(all->depth.end(), pr.depth.begin(), pr.depth.end());
        all->seq.insert(all->seq.end(), pr.seq.begin(), pr.seq.end());
        all->pts.insert(all->pts.end(), pr.pts.begin(), pr.pts.end());
        all->tau.insert(all->tau.end(), pr.tau.begin(), pr.tau.end());
    }
    return all;
}

// Diffuse reflection found by next-event estimation (Sec. II-F; the diffuse
// reflection of Sec. II-D).  Every launch ray (the canonical FP32 Fibonacci
// direction) bounces specularly as in sbr_ray, with its hit points
// s_b = o_b + t_b d_b and reflected directions kept in FP64.  At each of its hits
// s_j (j = 1..D) it is scattered diffusely towards every receiver that s_j sees,
// giving the path Tx -> s_1 .. s_{j-1} (specular) -> s_j (diffuse) -> Rx.  The
// receiver must lie strictly on the side of the plane of t_j from which the ray
// came (the side of s_{j-1}, or of the transmitter for j = 1), be farther than
// eps from s_j, and the segment s_j -> Rx must be free of every triangle but t_j
// for t in (eps, len - eps).  Paths are grouped by receiver and ordered by
// (ray, j) within a receiver; tau = (d_1 + .. + d_j + |Rx - s_j|) / c.
void* orc_diffuse_paths(void* h, const double* tx, const double* rx, int n_rx, int64_t n_rays, int D) {
    const Scene& s = *(Scene*)h;
    const double eps = 1e-6 * s.diag;
    const Vec3 txv = v3(tx[0], tx[1], tx[2]);
    std::vector<int32_t> seq((size_t)n_rays * D, -1);
    std::vector<Vec3> hit((size_t)n_rays * D);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n_rays; ++i) {
        float f[3];
        fibonacci_dir(i, n_rays, f);
        Vec3 o = txv, d = v3(f[0], f[1], f[2]);
        int prev = -1;
        for (int b = 0; b < D; ++b) {
            double th;
            int t = closest_hit(s, o, d, eps, prev, true, &th);
            if (t < 0) break;
            Vec3 p = o + th * d;
            seq[(size_t)D * i + b] = t;
            hit[(size_t)D * i + b] = p;
            Vec3 nn = s.n[t];
            d = d - (2.0 * dot(d, nn)) * nn;
            o = p;
            prev = t;
        }
    }
    std::vector<Paths> per_rx(n_rx);
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < n_rx; ++r) {
        const Vec3 rxv = v3(rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]);
        Paths& pr = per_rx[r];
        for (int64_t i = 0; i < n_rays; ++i) {
            double ell = 0.0;
            Vec3 prev_pt = txv;
            for (int j = 1; j <= D; ++j) {
                const int t = seq[(size_t)D * i + j - 1];
                if (t < 0) break;
                const Vec3 p = hit[(size_t)D * i + j - 1];
                ell += norm(p - prev_pt);
                const Vec3 nn = s.n[t];
                const double side_in = dot(prev_pt - p, nn), side_rx = dot(rxv - p, nn);
                const Vec3 seg = rxv - p;
                const double len = norm(seg);
                const bool same_side = (side_in > 0.0 && side_rx > 0.0) || (side_in < 0.0 && side_rx < 0.0);
                if (same_side && len > eps && !any_hit(s, p, seg, eps / len, 1.0 - eps / len, t, -1)) {
                    pr.rx.push_back(r);
                    pr.ray.push_back((int32_t)i);
                    pr.depth.push_back(j);
                    for (int b = 0; b < D; ++b) pr.seq.push_back(b < j ? seq[(size_t)D * i + b] : -1);
                    for (int k = 0; k < D + 2; ++k) {
                        Vec3 q = k == 0 ? txv : (k <= j ? hit[(size_t)D * i + k - 1] : (k == j + 1 ? rxv : v3(0, 0, 0)));
                        pr.pts.push_back(q.x);
                        pr.pts.push_back(q.y);
                        pr.pts.push_back(q.z);
                    }
                    pr.tau.push_back((ell + len) / kC0);
                }
                prev_pt = p;
            }
        }
    }
    Paths* all = new Paths();
    all->Dmax = D;
    for (int r = 0; r < n_rx; ++r) {
        Paths& pr = per_rx[r];
        all->rx.insert(all->rx.end(), pr.rx.begin(), pr.rx.end());
        all->ray.insert(all->ray.end(), pr.ray.begin(), pr.ray.end());
        all->depth.insert(all->depth.end(), pr.depth.begin(), pr.depth.end());
        all->seq.insert(all->seq.end(), pr.seq.begin(), pr.seq.end());
        all->pts.insert(all->pts.end(), pr.pts.begin(), pr.pts.end());
        all->tau.insert(all->tau.end(), pr.tau.begin(), pr.tau.end());
    }
    return all;
}

void orc_paths_rays(void* p, int32_t* ray) {
    Paths& P = *(Paths*)p;
    std::memcpy(ray, P.ray.data(), sizeof(int32_t) * P.ray.size());
}

int64_t orc_paths_count(void* p) { return (int64_t)((Paths*)p)->depth.size(); }

void orc_paths_get(void* p, int32_t* rx, int32_t* depth, int32_t* seq, double* pts, double* tau) {
    Paths& P = *(Paths*)p;
    std::memcpy(rx, P.rx.data(), sizeof(int32_t) * P.rx.size());
    std::memcpy(depth, P.depth.data(), sizeof(int32_t) * P.depth.size());
    std::memcpy(seq, P.seq.data(), sizeof(int32_t) * P.seq.size());
    std::memcpy(pts, P.pts.data(), sizeof(double) * P.pts.size());
    std::memcpy(tau, P.tau.data(), sizeof(double) * P.tau.size());
}

void orc_paths_free(void* p) { delete (Paths*)p; }

// Path coefficients a_i (interleaved re/im) of P paths given by their points.
// seq: P x Dmax, pts: P x (Dmax+2) x 3 (Tx, s_1..s_q, Rx, padding).
void orc_fields(void* h, int64_t P, int Dmax, const int32_t* depth, const int32_t* seq, const double* pts,
                const int32_t* tri_material, const float* eps_r, const float* sigma, const uint8_t* is_pec,
                int per_triangle, double freq, double gain_tx, double gain_rx, int ni_mode, double* a_out) {
    const Scene& s = *(Scene*)h;
    PathMaterials m{tri_material, eps_r, sigma, is_pec, per_triangle};
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < P; ++i) {
        int q = depth[i];
        std::vector<Vec3> pv(q + 2);
        for (int j = 0; j <= q; ++j) {
            const double* p = pts + ((size_t)(Dmax + 2) * i + j) * 3;
            pv[j] = v3(p[0], p[1], p[2]);
        }
        const double* pr = pts + ((size_t)(Dmax + 2) * i + q + 1) * 3;
        pv[q + 1] = v3(pr[0], pr[1], pr[2]);
        ChainOut co;
        path_chain(s, m, pv.data(), seq + (size_t)Dmax * i, q, freq, gain_tx, gain_rx, ni_mode, &co);
        a_out[2 * i] = co.a.real();
        a_out[2 * i + 1] = co.a.imag();
    }
}

// Gradients of a real loss L given g_a = dL/dRe a + j dL/dIm a for every path:
// dL/dx = Re(conj(g_a) da/dx).  With eta = eps_r - j sigma/(eps0 omega):
// da/deps_r = da/deta, da/dsigma = -j/(eps0 omega) da/deta, da/dg_T = a/(2 g_T),
// da/dg_R = a/(2 g_R).  Results are accumulated into the outputs.
void orc_fields_grad(void* h, int64_t P, int Dmax, const int32_t* depth, const int32_t* seq, const double* pts,
                     const int32_t* tri_material, const float* eps_r, const float* sigma, const uint8_t* is_pec,
                     int per_triangle, double freq, double gain_tx, double gain_rx, const double* grad_a,
                     double* grad_eps, double* grad_sigma, double* grad_gain) {
    const Scene& s = *(Scene*)h;
    PathMaterials m{tri_material, eps_r, sigma, is_pec, per_triangle};
    const cplx deta_dsigma(0.0, -1.0 / (kEps0 * 2.0 * kPi * freq));
    for (int64_t i = 0; i < P; ++i) {
        int q = depth[i];
        std::vector<Vec3> pv(q + 2);
        for (int j = 0; j <= q; ++j) {
            const double* p = pts + ((size_t)(Dmax + 2) * i + j) * 3;
            pv[j] = v3(p[0], p[1], p[2]);
        }
        const double* pr = pts + ((size_t)(Dmax + 2) * i + q + 1) * 3;
        pv[q + 1] = v3(pr[0], pr[1], pr[2]);
        ChainOut co;
        path_chain(s, m, pv.data(), seq + (size_t)Dmax * i, q, freq, gain_tx, gain_rx, 0, &co);
        cplx g(grad_a[2 * i], grad_a[2 * i + 1]);
        for (int j = 0; j < q; ++j) {
            if (co.pec[j]) continue;
            grad_eps[co.mat[j]] += (std::conj(g) * co.da_deta[j]).real();
            grad_sigma[co.mat[j]] += (std::conj(g) * co.da_deta[j] * deta_dsigma).real();
        }
        grad_gain[0] += (std::conj(g) * co.a).real() / (2.0 * gain_tx);
        grad_gain[1] += (std::conj(g) * co.a).real() / (2.0 * gain_rx);
    }
}

// Discrete CFR (Sec. II-A): H[r, n] = sum_{i in r} a_i exp(-j 2 pi (f_c + n df) tau_i),
// n = -N/2 .. N/2-1, stored at column n + N/2.  a, H interleaved re/im.
void orc_cfr(int64_t P, const double* a, const double* tau, const int64_t* rx_offsets, int n_rx, double fc,
             double df, int N, double* H) {
    (void)P;
#pragma omp parallel for schedule(dynamic, 4)
    for (int r = 0; r < n_rx; ++r) {
        for (int c = 0; c < N; ++c) {
            double f = fc + (double)(c - N / 2) * df;
            cplx acc = 0.0;
            for (int64_t i = rx_offsets[r]; i < rx_offsets[r + 1]; ++i)
                acc += cplx(a[2 * i], a[2 * i + 1]) * std::polar(1.0, -2.0 * kPi * f * tau[i]);
            H[2 * ((size_t)r * N + c)] = acc.real();
            H[2 * ((size_t)r * N + c) + 1] = acc.imag();
        }
    }
}

// Adjoint of orc_cfr: g_a[i] = sum_n g_H[r(i), n] conj(exp(-j 2 pi f_n tau_i)).
void orc_cfr_grad(int64_t P, const double* tau, const int64_t* rx_offsets, int n_rx, double fc, double df, int N,
                  const double* grad_H, double* grad_a) {
    (void)P;
#pragma omp parallel for schedule(dynamic, 4)
    for (int r = 0; r < n_rx; ++r) {
        for (int64_t i = rx_offsets[r]; i < rx_offsets[r + 1]; ++i) {
            cplx acc = 0.0;
            for (int c = 0; c < N; ++c) {
                double f = fc + (double)(c - N / 2) * df;
                cplx g(grad_H[2 * ((size_t)r * N + c)], grad_H[2 * ((size_t)r * N + c) + 1]);
                acc += g * std::conj(std::polar(1.0, -2.0 * kPi * f * tau[i]));
            }
            grad_a[2 * i] = acc.real();
            grad_a[2 * i + 1] = acc.imag();
        }
    }
}

// ---------------------------------------------------------------------------
// First-order diffraction (Sec. II-D, Eq. diffraction; candidates and the point of
// diffraction, Sec. II-F).  The paper models edges as infinitely long wedges
// whose two faces may carry different materials, takes candidate edges from the
// shoot-and-bouncing rays and finds the point of diffraction by Keller's
// principle of the shortest path.  Readings (the paper is silent on them):
//  * Wedges.  Triangles share an edge when two of their vertices coincide in
//    position.  An edge shared by exactly two triangles is a wedge when its exterior
//    angle n pi (measured outside the solid, between the two faces, from the
//    triangles' winding normals taken as outward) has 1 < n <= 2; n = 2 is a
//    screen (two coincident faces back to back).  A flat pair (n = 1), a concave
//    pair (n < 1), a border edge (one triangle), an edge of three or more triangles
//    and a pair with inconsistent winding are not wedges.  The geometry is taken
//    literally (a box standing on a ground plane keeps its base edges).
//  * Canonical frame of a wedge: face 0 is the lower triangle index, t0 the unit
//    vector from the edge into face 0, n0 its normal, e = t0 x n0 the edge
//    direction, so that angles about e grow from face 0 into the exterior; the
//    edge runs from its start vertex E_s to E_s + l e.
//  * Candidate wedges: those with a face among the triangles that the launch rays
//    hit first (the depth-1 candidates of the specular trace).
//  * Point of diffraction Q: on the edge line, the point minimising |Tx - Q| +
//    |Q - Rx| (Keller), x_Q = (x_T b + x_R a) / (a + b) along e from E_s, with a, b
//    the distances of Tx and Rx from the line and x_T, x_R their abscissae.  Valid
//    when a, b > eps, 0 <= x_Q < l (half-open, so a point shared by collinear edge
//    pieces belongs to one of them), Tx and Rx lie strictly in the exterior
//    (0 < phi', phi < n pi), |Q - Tx|, |Rx - Q| > eps, and both segments are free
//    of triangles other than the two faces for t in (eps, len - eps).
//  * Incidence face (Luebbers' R_0): the face on the transmitter's side, i.e. the
//    labels are swapped when the transmitter's angle phi' exceeds n pi / 2.
struct Wedge {
    int f0, fn;          // canonical: f0 < fn
    Vec3 es, e, t0, n0;  // start vertex, edge direction, face-0 frame
    double len, n;
};

static bool vless(Vec3 a, Vec3 b) {
    if (a.x != b.x) return a.x < b.x;
    if (a.y != b.y) return a.y < b.y;
    return a.z < b.z;
}

static std::vector<Wedge> build_wedges(const Scene& s) {
    std::map<std::array<double, 6>, std::vector<int>> edges;
    for (int t = 0; t < s.T; ++t) {
        Vec3 v[3] = {s.a[t], s.b[t], s.c[t]};
        for (int k = 0; k < 3; ++k) {
            Vec3 p = v[k], q = v[(k + 1) % 3];
            if (vless(q, p)) std::swap(p, q);
            edges[{p.x, p.y, p.z, q.x, q.y, q.z}].push_back(t);
        }
    }
    std::vector<Wedge> out;
    for (auto& kv : edges) {
        if (kv.second.size() != 2) continue;
        int f0 = std::min(kv.second[0], kv.second[1]), f1 = std::max(kv.second[0], kv.second[1]);
        if (f0 == f1) continue;
        Vec3 A = v3(kv.first[0], kv.first[1], kv.first[2]), B = v3(kv.first[3], kv.first[4], kv.first[5]);
        Vec3 er = unit(B - A);
        auto inward = [&](int t) {   // unit vector from the edge into triangle t, normal to the edge
            Vec3 v[3] = {s.a[t], s.b[t], s.c[t]};
            Vec3 c = v[0];
            for (int k = 0; k < 3; ++k)
                if (!((v[k].x == A.x && v[k].y == A.y && v[k].z == A.z) || (v[k].x == B.x && v[k].y == B.y && v[k].z == B.z)))
                    c = v[k];
            Vec3 w = c - A;
            return unit(w - dot(w, er) * er);
        };
        Vec3 t0 = inward(f0), t1 = inward(f1);
        Vec3 n0 = s.n[f0], n1 = s.n[f1];
        Vec3 e = dot(cross(er, t0), n0) >= 0.0 ? er : -1.0 * er;
        // face n must face the exterior too: its normal is -(e x t1)
        if (dot(-1.0 * cross(e, t1), n1) <= 0.5) continue;
        double psi = std::atan2(dot(t1, n0), dot(t1, t0));
        if (psi < 0.0) psi += 2.0 * kPi;
        if (psi < 1e-12) psi = 2.0 * kPi;   // coincident faces back to back: a screen
        double n = psi / kPi;
        if (!(n > 1.0 + 1e-9)) continue;
        Wedge w;
        w.f0 = f0;
        w.fn = f1;
        w.e = e;
        w.t0 = t0;
        w.n0 = n0;
        w.len = norm(B - A);
        w.es = dot(B - A, e) > 0.0 ? A : B;
        w.n = n;
        out.push_back(w);
    }
    std::sort(out.begin(), out.end(), [](const Wedge& x, const Wedge& y) {
        return x.f0 != y.f0 ? x.f0 < y.f0 : x.fn < y.fn;
    });
    return out;
}

// angle of direction d about the wedge's edge, from face 0 towards the exterior, in [0, 2 pi)
static double wedge_angle(const Wedge& w, Vec3 d) {
    Vec3 p = d - dot(d, w.e) * w.e;
    double a = std::atan2(dot(p, w.n0), dot(p, w.t0));
    return a < 0.0 ? a + 2.0 * kPi : a;
}

struct WedgeTable {
    std::vector<Wedge> w;
};

void* orc_wedges(void* h) {
    WedgeTable* t = new WedgeTable();
    t->w = build_wedges(*(Scene*)h);
    return t;
}

int64_t orc_wedges_count(void* wt) { return (int64_t)((WedgeTable*)wt)->w.size(); }

// per wedge: faces (f0, fn), start vertex, edge direction, t0, n0 (3 each), length, n
void orc_wedges_get(void* wt, int32_t* faces, double* geo) {
    const std::vector<Wedge>& W = ((WedgeTable*)wt)->w;
    for (size_t i = 0; i < W.size(); ++i) {
        faces[2 * i] = W[i].f0;
        faces[2 * i + 1] = W[i].fn;
        double* g = geo + 14 * i;
        Vec3 v[4] = {W[i].es, W[i].e, W[i].t0, W[i].n0};
        for (int k = 0; k < 4; ++k) {
            g[3 * k] = v[k].x;
            g[3 * k + 1] = v[k].y;
            g[3 * k + 2] = v[k].z;
        }
        g[12] = W[i].len;
        g[13] = W[i].n;
    }
}

void orc_wedges_free(void* wt) { delete (WedgeTable*)wt; }

// Diffraction paths Tx -> Q -> Rx for every (candidate wedge, receiver).  Output
// (Paths, Dmax = 2, depth 1): seq = (incidence face, other face), pts = Tx, Q, Rx,
// plus `ray` = the wedge's index in the wedge table; grouped by receiver, by wedge
// within a receiver.
void* orc_diffraction_paths(void* h, void* wt, const double* tx, const double* rx, int n_rx, void* cand_h) {
    const Scene& s = *(Scene*)h;
    const std::vector<Wedge>& W = ((WedgeTable*)wt)->w;
    std::vector<int32_t>& cv = *(std::vector<int32_t>*)cand_h;
    const int D = cv[0];
    const int64_t K = cv[1];
    std::vector<char> first(s.T, 0);
    for (int64_t k = 0; k < K; ++k) {
        const int32_t* sq = cv.data() + 2 + (size_t)D * k;
        if (sq[0] >= 0 && (D == 1 || sq[1] < 0)) first[sq[0]] = 1;
    }
    std::vector<int> cw;
    for (size_t i = 0; i < W.size(); ++i)
        if (first[W[i].f0] || first[W[i].fn]) cw.push_back((int)i);
    const double eps = 1e-6 * s.diag;
    const Vec3 T = v3(tx[0], tx[1], tx[2]);
    std::vector<Paths> per(n_rx);
#pragma omp parallel for schedule(dynamic, 4)
    for (int r = 0; r < n_rx; ++r) {
        const Vec3 R = v3(rx[3 * r], rx[3 * r + 1], rx[3 * r + 2]);
        Paths& pr = per[r];
        for (int wi : cw) {
            const Wedge& w = W[wi];
            double xT = dot(T - w.es, w.e), xR = dot(R - w.es, w.e);
            double a = norm(T - w.es - xT * w.e), b = norm(R - w.es - xR * w.e);
            if (!(a > eps && b > eps)) continue;
            double xQ = (xT * b + xR * a) / (a + b);
            if (!(xQ >= 0.0 && xQ < w.len)) continue;
            Vec3 Q = w.es + xQ * w.e;
            double php = wedge_angle(w, T - Q), ph = wedge_angle(w, R - Q);
            double lim = w.n * kPi;
            if (!(php > 0.0 && php < lim && ph > 0.0 && ph < lim)) continue;
            double sp = norm(Q - T), sd = norm(R - Q);
            if (!(sp > eps && sd > eps)) continue;
            if (any_hit(s, T, Q - T, eps / sp, 1.0 - eps / sp, w.f0, w.fn)) continue;
            if (any_hit(s, Q, R - Q, eps / sd, 1.0 - eps / sd, w.f0, w.fn)) continue;
            bool swap = php > 0.5 * lim;
            pr.depth.push_back(1);
            pr.seq.push_back(swap ? w.fn : w.f0);
            pr.seq.push_back(swap ? w.f0 : w.fn);
            for (Vec3 p : {T, Q, R, v3(0, 0, 0)}) {
                pr.pts.push_back(p.x);
                pr.pts.push_back(p.y);
                pr.pts.push_back(p.z);
            }
            pr.tau.push_back((sp + sd) / kC0);
            pr.ray.push_back(wi);
        }
    }
    Paths* all = new Paths();
    all->Dmax = 2;
    for (int r = 0; r < n_rx; ++r) {
        Paths& pr = per[r];
        for (size_t i = 0; i < pr.depth.size(); ++i) all->rx.push_back(r);
        all->depth.insert(all->depth.end(), pr.depth.begin(), pr.depth.end());
        all->seq.insert(all->seq.end(), pr.seq.begin(), pr.seq.end());
        all->pts.insert(all->pts.end(), pr.pts.begin(), pr.pts.end());
        all->tau.insert(all->tau.end(), pr.tau.begin(), pr.tau.end());
        all->ray.insert(all->ray.end(), pr.ray.begin(), pr.ray.end());
    }
    return all;
}

void orc_fresnel(double eps_r, double sigma, double freq, double cos_i, double* out) {
    cplx rp, rl;
    fresnel(permittivity(eps_r, sigma, freq), cos_i, &rp, &rl);
    out[0] = rp.real(); out[1] = rp.imag(); out[2] = rl.real(); out[3] = rl.imag();
    cplx dp, dl;
    fresnel_deta(permittivity(eps_r, sigma, freq), cos_i, &dp, &dl);
    out[4] = dp.real(); out[5] = dp.imag(); out[6] = dl.real(); out[7] = dl.imag();
}

void orc_permittivity(double eps_r, double sigma, double freq, double* out) {
    cplx e = permittivity(eps_r, sigma, freq);
    out[0] = e.real();
    out[1] = e.imag();
}

}  // extern "C"
