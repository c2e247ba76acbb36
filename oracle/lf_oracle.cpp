// FP64 brute-force oracle for 2D-Gaussian surfel ray tracing with one-bounce
// physically based shading under an environment map.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
// CUDA path is checked against.  Only the test suite, the smoke check and the
// CPU-baseline leg of the benchmark may load it.  It shares no code, header,
// table or constant generator with the CUDA library.
//
// What it computes, step by step, in the paper's order:
//   * Eq. 6: every ray is intersected with the plane of EVERY surfel (no
//     acceleration structure); the hit is projected on the tangent axes to
//     xi = (u, v); alpha~ = min(0.99, o exp(-|xi|^2/2)); hits outside the
//     support (u^2+v^2 > R^2) or under the opacity threshold are dropped.
//   * The accepted hits are FULLY sorted by the key (t, surfel id).
//   * Eq. 7: front-to-back compositing T_j, w_j = T_j alpha_j,
//     z_bar = sum w z / (sum w + eps) for position, depth, normal and
//     material; the normal is renormalised.  Compositing stops after the hit
//     whose transmittance falls below T_min.
//   * Eq. 10-11 with the per-sample budget of Sec. 4.2: one environment
//     next-event sample at the primary record, one BSDF continuation drawn
//     from a cosine/GGX mixture, at most one secondary record, two environment
//     samples there; power-heuristic MIS between the primary NEE and the BSDF
//     continuation.  Metallic-roughness BRDF: Lambert + GGX (Walter et al.
//     2007), separable Smith G, Schlick Fresnel.
//   * Sec. 3.3 (path replay): the gradient treats the sampled directions,
//     pdfs, MIS weights, visibilities and the whole secondary record as
//     constants; it flows through the primary record (Eq. 6-7 -> surfel
//     parameters), the primary transmittance and every environment lookup.
//     The gradient is taken by a small FP64 reverse-mode tape over the very
//     same templated code that computes the forward value.
//   * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
//     counter = (pixel, sample, group, 0), key = (seed lo, seed hi).
//
// Readings of points the paper leaves open (support radius, thresholds, eps,
// stop rule, env mapping, lobe probability, ...) come in through or_params.
// The environment importance sampler works on the FP64 tables throughout: the
// texel a uniform selects and its position inside the texel.  Where a uniform
// sits within FP32 rounding of a CDF entry (a renderer with FP32 tables may
// pick the neighbouring texel) the sample records a margin and is flagged.
//
// Compile (see oracle/__init__.py):  g++ -O2 -fopenmp -ffp-contract=off -shared -fPIC

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <unordered_map>
#include <vector>
#include <omp.h>

namespace {

const double PI = 3.14159265358979323846;

// ------------------------------------------------------------------------
// Philox4x32-10 (SC'11): 10 rounds of two 32x32->64 multiplies, Weyl key bump.
// ------------------------------------------------------------------------
void philox4x32_10(const uint32_t in[4], uint32_t k0, uint32_t k1, uint32_t out[4]) {
  uint32_t c0 = in[0], c1 = in[1], c2 = in[2], c3 = in[3];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

inline double to_unit(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

// Sobol direction numbers for 9 dimensions (Joe and Kuo 2008: primitive
// polynomial of degree s with coefficients a, initial numbers m; the first
// dimension is van der Corput), as 32-bit fractions from the recurrence
//   v_k = m_k 2^(31-k) (k < s),  v_k = v_{k-s} xor (v_{k-s} >> s) xor (xor over j < s with bit a_j: v_{k-j}).
struct SobolTable {
  uint32_t v[9][32];
  SobolTable() {
    const int deg[9] = {0, 1, 2, 3, 3, 4, 4, 5, 5};
    const int coef[9] = {0, 0, 1, 1, 2, 1, 4, 2, 4};
    const uint32_t init[9][5] = {{1}, {1}, {1, 3}, {1, 3, 1}, {1, 1, 1}, {1, 1, 3, 3}, {1, 3, 5, 13},
                                 {1, 1, 5, 5, 17}, {1, 1, 5, 5, 5}};
    for (int k = 0; k < 32; ++k) v[0][k] = 1u << (31 - k);
    for (int d = 1; d < 9; ++d)
      for (int k = 0; k < 32; ++k) {
        const int s = deg[d];
        if (k < s) { v[d][k] = init[d][k] << (31 - k); continue; }
        uint32_t x = v[d][k - s] ^ (v[d][k - s] >> s);
        for (int j = 1; j < s; ++j)
          if ((coef[d] >> (s - 1 - j)) & 1) x ^= v[d][k - j];
        v[d][k] = x;
      }
  }
};
const SobolTable& sobol_table() {
  static const SobolTable t;
  return t;
}
// Point `index` of Sobol dimension d: XOR of the direction numbers of its set bits.
uint32_t sobol32(uint32_t index, int d) {
  uint32_t x = 0;
  for (int k = 0; index; ++k, index >>= 1)
    if (index & 1u) x ^= sobol_table().v[d][k];
  return x;
}

// The nine uniforms of one (pixel, sample): NEE (0,1), lobe 2, BSDF (3,4),
// secondary NEE #1 (5,6), secondary NEE #2 (7,8).
//  sampler 0: Philox4x32-10 of counter (pixel, sample, group, 0), groups 0-2;
//  sampler 1: the Sobol point of index `sample`, rotated modulo 1 per pixel by
//             Philox4x32-10 of counter (pixel, 0xffffffff, group, 1), in 24-bit
//             fixed point.
void sample_uniforms(uint32_t pixel, uint32_t sample, uint64_t seed, int sampler, double u[9]) {
  uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
  uint32_t out[4];
  for (uint32_t g = 0; g < 3; ++g) {
    uint32_t ctr[4] = {pixel, sampler == 1 ? 0xffffffffu : sample, g, sampler == 1 ? 1u : 0u};
    philox4x32_10(ctr, k0, k1, out);
    for (int i = 0; i < 4; ++i) {
      const int idx = (int)g * 4 + i;
      if (idx >= 9) continue;
      if (sampler == 1) {
        const uint32_t x = ((sobol32(sample, idx) >> 8) + (out[i] >> 8)) & 0xffffffu;
        u[idx] = (double)x * (1.0 / 16777216.0);
      } else {
        u[idx] = to_unit(out[i]);
      }
    }
  }
}

// ------------------------------------------------------------------------
// Reverse-mode tape.
// ------------------------------------------------------------------------
struct TNode { int a, b; double da, db; };
struct Tape {
  std::vector<TNode> nodes;
  int push(int a, double da, int b, double db) {
    nodes.push_back({a, b, da, db});
    return (int)nodes.size() - 1;
  }
};
thread_local Tape* g_tape = nullptr;

struct Var {
  double v;
  int id;
  Var() : v(0.0), id(-1) {}
  Var(double x) : v(x), id(-1) {}  // NOLINT: constants convert implicitly
};

inline int rec2(int a, double da, int b, double db) {
  if (a < 0 && b < 0) return -1;
  return g_tape->push(a, da, b, db);
}
inline Var mk(double v, int id) { Var r; r.v = v; r.id = id; return r; }
inline Var make_input(double v) { return mk(v, g_tape->push(-1, 0.0, -1, 0.0)); }

inline Var operator+(const Var& x, const Var& y) { return mk(x.v + y.v, rec2(x.id, 1.0, y.id, 1.0)); }
inline Var operator-(const Var& x, const Var& y) { return mk(x.v - y.v, rec2(x.id, 1.0, y.id, -1.0)); }
inline Var operator*(const Var& x, const Var& y) { return mk(x.v * y.v, rec2(x.id, y.v, y.id, x.v)); }
inline Var operator/(const Var& x, const Var& y) {
  double r = x.v / y.v;
  return mk(r, rec2(x.id, 1.0 / y.v, y.id, -r / y.v));
}
inline Var operator-(const Var& x) { return mk(-x.v, rec2(x.id, -1.0, -1, 0.0)); }
inline Var operator+(const Var& x, double y) { return mk(x.v + y, rec2(x.id, 1.0, -1, 0.0)); }
inline Var operator+(double x, const Var& y) { return y + x; }
inline Var operator-(const Var& x, double y) { return mk(x.v - y, rec2(x.id, 1.0, -1, 0.0)); }
inline Var operator-(double x, const Var& y) { return mk(x - y.v, rec2(y.id, -1.0, -1, 0.0)); }
inline Var operator*(const Var& x, double y) { return mk(x.v * y, rec2(x.id, y, -1, 0.0)); }
inline Var operator*(double x, const Var& y) { return y * x; }
inline Var operator/(const Var& x, double y) { return mk(x.v / y, rec2(x.id, 1.0 / y, -1, 0.0)); }
inline Var operator/(double x, const Var& y) {
  double r = x / y.v;
  return mk(r, rec2(y.id, -r / y.v, -1, 0.0));
}
inline Var& operator+=(Var& x, const Var& y) { x = x + y; return x; }
inline Var sqrt(const Var& x) {
  double r = std::sqrt(x.v);
  return mk(r, rec2(x.id, r > 0 ? 0.5 / r : 0.0, -1, 0.0));
}
inline Var exp(const Var& x) {
  double r = std::exp(x.v);
  return mk(r, rec2(x.id, r, -1, 0.0));
}

inline double val(double x) { return x; }
inline double val(const Var& x) { return x.v; }

template <class S> struct V3 {
  S x, y, z;
  V3() : x(0.0), y(0.0), z(0.0) {}
  V3(S a, S b, S c) : x(a), y(b), z(c) {}
};
template <class S> V3<S> operator+(const V3<S>& a, const V3<S>& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class S> V3<S> operator-(const V3<S>& a, const V3<S>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class S, class T> V3<S> scl(const V3<S>& a, const T& s) { return {a.x * s, a.y * s, a.z * s}; }
template <class S> V3<S> mul(const V3<S>& a, const V3<S>& b) { return {a.x * b.x, a.y * b.y, a.z * b.z}; }
template <class S> S dot(const V3<S>& a, const V3<S>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class S> V3<S> cross(const V3<S>& a, const V3<S>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class S> V3<S> lift(const V3<double>& a) { return {S(a.x), S(a.y), S(a.z)}; }

using D3 = V3<double>;
inline double norm(const D3& a) { return std::sqrt(dot(a, a)); }
// Division (not a multiply by the reciprocal) keeps the unit normal of an
// axis-aligned plane exact, so coplanar surfels get exactly equal depths.
inline D3 normalize(const D3& a) {
  const double l = norm(a);
  return {a.x / l, a.y / l, a.z / l};
}

// ------------------------------------------------------------------------
// Inputs.
// ------------------------------------------------------------------------
struct Params {
  double T_min, alpha_min, alpha_max, support_r2, eps_w, t_min, ray_offset, p_spec;
  int brdf_mode, sampling_mode, sampler;
};

struct SceneD {  // FP64 copy of the FP32 inputs plus the plane normal n^ of each surfel
  int n = 0;
  std::vector<D3> mu, tu, tv, nh, a;
  std::vector<double> su, sv, op, m, r;
};

// ------------------------------------------------------------------------
// Discontinuity margins (smallest distance of any decision that could change
// the result to its threshold), kept per ray group: the primary ray of a
// pixel, and each shading sample.
// ------------------------------------------------------------------------
// CDF: distance (in the uniform) of an environment sample's uniforms to the
// CDF entries that bound the selected texel.  PTEX: angular distance (in
// radians) of a continuation direction to the texel edges of the
// piecewise-constant environment pdf that its MIS weight reads.
// SUPPORT_SHIFT, ALPHA_SHIFT, TIE_SHIFT: the support, opacity-threshold and
// depth-order decisions again, measured as the shift of the ray (world
// units, first order, a change of direction counted as (1 + t) times one of
// the origin) that flips them: a shading ray that starts from another
// rounding of the same composite moves by such a shift.
enum { M_SUPPORT, M_ALPHA, M_CAP, M_TMIN, M_TIE, M_STOP, M_COS, M_FRAME, M_CDF, M_PTEX, M_SUPPORT_SHIFT,
       M_ALPHA_SHIFT, M_TIE_SHIFT, NMARGIN };
struct Margins {
  double m[NMARGIN];
  Margins() { for (double& x : m) x = std::numeric_limits<double>::infinity(); }
  void put(int k, double v) { m[k] = std::min(m[k], std::fabs(v)); }
  void merge(const Margins& o) { for (int k = 0; k < NMARGIN; ++k) m[k] = std::min(m[k], o.m[k]); }
};

struct Env {
  int H = 0, W = 0;
  const float* rgb = nullptr;        // (H, W, 3) lookups (live values)
  std::vector<double> pmf_row, cdf_row, pmf_col, cdf_col;  // sampling tables (FP64)
};

// Sampling tables: texel weight = (Rec.709 luminance + 1e-6) * sin(theta at the
// row centre); marginal over rows, conditional over columns; sequential FP64
// prefix sums; the last CDF entry of each table is exactly 1.
void build_env_tables(Env& e) {
  const int H = e.H, W = e.W;
  std::vector<double> w((size_t)H * W), rowsum(H);
  for (int r = 0; r < H; ++r) {
    double st = std::sin(PI * ((double)r + 0.5) / (double)H);
    double acc = 0.0;
    for (int c = 0; c < W; ++c) {
      const float* t = e.rgb + ((size_t)r * W + c) * 3;
      double lum = 0.2126 * (double)t[0] + 0.7152 * (double)t[1];
      lum = lum + 0.0722 * (double)t[2];
      lum = lum + 1e-6;
      w[(size_t)r * W + c] = lum * st;
    }
    for (int c = 0; c < W; ++c) acc = acc + w[(size_t)r * W + c];
    rowsum[r] = acc;
  }
  double total = 0.0;
  for (int r = 0; r < H; ++r) total = total + rowsum[r];
  e.pmf_row.assign(H, 0.0); e.cdf_row.assign(H, 0.0);
  e.pmf_col.assign((size_t)H * W, 0.0); e.cdf_col.assign((size_t)H * W, 0.0);
  double pre = 0.0;
  for (int r = 0; r < H; ++r) {
    pre = pre + rowsum[r];
    e.pmf_row[r] = rowsum[r] / total;
    e.cdf_row[r] = pre / total;
    double pc = 0.0;
    for (int c = 0; c < W; ++c) {
      pc = pc + w[(size_t)r * W + c];
      e.pmf_col[(size_t)r * W + c] = w[(size_t)r * W + c] / rowsum[r];
      e.cdf_col[(size_t)r * W + c] = pc / rowsum[r];
    }
  }
}

// y-up equirectangular mapping: theta = acos(w_y), phi = atan2(w_x, -w_z) + pi.
inline void dir_to_angles(const D3& w, double& th, double& ph) {
  th = std::acos(std::max(-1.0, std::min(1.0, w.y)));
  ph = std::atan2(w.x, -w.z) + PI;
}
inline D3 angles_to_dir(double th, double ph) {
  double s = std::sin(th), p = ph - PI;
  return {s * std::sin(p), std::cos(th), -s * std::cos(p)};
}

// First index i in [0,n) with f[i] > u (f non-decreasing, f[n-1] == 1 > u).
int first_greater(const double* f, int n, double u) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi) / 2;
    if (f[mid] > u) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// Texel (row, column) of a direction in the piecewise-constant pdf; with a
// margin sink, also the angular distance of the direction to the nearest
// texel edge (the row edges at the poles are not decisions).
void pdf_texel(const Env& e, const D3& w, int& r, int& c, double& th, Margins* mg) {
  double ph;
  dir_to_angles(w, th, ph);
  const double y = th / PI * e.H, x = ph / (2 * PI) * e.W;
  r = std::min(e.H - 1, std::max(0, (int)std::floor(y)));
  c = std::min(e.W - 1, std::max(0, (int)std::floor(x)));
  if (mg) {
    if (y > 0.5 && y < e.H - 0.5) mg->put(M_PTEX, (y - std::nearbyint(y)) * PI / e.H);
    mg->put(M_PTEX, (x - std::nearbyint(x)) * 2.0 * PI / e.W * std::sin(th));
  }
}

double env_pdf(const Env& e, const D3& w, Margins* mg = nullptr) {
  int r, c;
  double th;
  pdf_texel(e, w, r, c, th, mg);
  double st = std::max(std::sin(th), 1e-12);
  return e.pmf_row[r] * e.pmf_col[(size_t)r * e.W + c] * (double)e.H * (double)e.W / (2.0 * PI * PI * st);
}

// Inverse-CDF sample of the piecewise-constant environment density: the row
// from the marginal table, the column from that row's conditional table,
// uniform inside the texel.  Margin: distance of each uniform to the CDF
// entries that bound its choice.
void env_sample(const Env& e, double u1, double u2, D3& w, double& pdf, Margins* mg = nullptr) {
  int r = first_greater(e.cdf_row.data(), e.H, u1);
  double lo = r > 0 ? e.cdf_row[r - 1] : 0.0, hi = e.cdf_row[r];
  double fr = std::min(std::max((u1 - lo) / (hi - lo), 0.0), 1.0);
  const double* row = e.cdf_col.data() + (size_t)r * e.W;
  int c = first_greater(row, e.W, u2);
  double clo = c > 0 ? row[c - 1] : 0.0, chi = row[c];
  double fc = std::min(std::max((u2 - clo) / (chi - clo), 0.0), 1.0);
  if (mg) {
    if (r > 0) mg->put(M_CDF, u1 - lo);
    if (r < e.H - 1) mg->put(M_CDF, hi - u1);
    if (c > 0) mg->put(M_CDF, u2 - clo);
    if (c < e.W - 1) mg->put(M_CDF, chi - u2);
  }
  double th = PI * ((double)r + fr) / (double)e.H;
  double ph = 2.0 * PI * ((double)c + fc) / (double)e.W;
  w = angles_to_dir(th, ph);
  double st = std::max(std::sin(th), 1e-12);
  pdf = e.pmf_row[r] * e.pmf_col[(size_t)r * e.W + c] * (double)e.H * (double)e.W / (2.0 * PI * PI * st);
}

// Bilinear weights of the lookup E(w): four texels, u wraps, v clamps.
struct Bilin { int idx[4]; double wt[4]; };
Bilin env_bilinear(const Env& e, const D3& w) {
  double th, ph;
  dir_to_angles(w, th, ph);
  double u = ph / (2.0 * PI) * e.W - 0.5, v = th / PI * e.H - 0.5;
  double x0f = std::floor(u), y0f = std::floor(v);
  double fx = u - x0f, fy = v - y0f;
  long x0 = (long)x0f, y0 = (long)y0f;
  long x0m = ((x0 % e.W) + e.W) % e.W, x1m = (((x0 + 1) % e.W) + e.W) % e.W;
  long y0c = std::min<long>(e.H - 1, std::max<long>(0, y0)), y1c = std::min<long>(e.H - 1, std::max<long>(0, y0 + 1));
  Bilin b;
  b.idx[0] = (int)(y0c * e.W + x0m); b.wt[0] = (1 - fx) * (1 - fy);
  b.idx[1] = (int)(y0c * e.W + x1m); b.wt[1] = fx * (1 - fy);
  b.idx[2] = (int)(y1c * e.W + x0m); b.wt[2] = (1 - fx) * fy;
  b.idx[3] = (int)(y1c * e.W + x1m); b.wt[3] = fx * fy;
  return b;
}

// Environment providers: plain values, or tape inputs (one per texel channel).
struct EnvValues {
  const Env* e;
  V3<double> lookup(const D3& w) {
    Bilin b = env_bilinear(*e, w);
    V3<double> s;
    for (int k = 0; k < 4; ++k) {
      const float* t = e->rgb + (size_t)b.idx[k] * 3;
      s.x = s.x + b.wt[k] * (double)t[0];
      s.y = s.y + b.wt[k] * (double)t[1];
      s.z = s.z + b.wt[k] * (double)t[2];
    }
    return s;
  }
};
struct EnvTape {
  const Env* e;
  std::unordered_map<int, int> texel_var;  // texel -> id of its R input (G, B follow)
  V3<Var> lookup(const D3& w) {
    Bilin b = env_bilinear(*e, w);
    V3<Var> s;
    for (int k = 0; k < 4; ++k) {
      auto it = texel_var.find(b.idx[k]);
      int base;
      const float* t = e->rgb + (size_t)b.idx[k] * 3;
      if (it == texel_var.end()) {
        base = make_input(t[0]).id;
        make_input(t[1]);
        make_input(t[2]);
        texel_var[b.idx[k]] = base;
      } else {
        base = it->second;
      }
      s.x = s.x + mk(t[0], base) * b.wt[k];
      s.y = s.y + mk(t[1], base + 1) * b.wt[k];
      s.z = s.z + mk(t[2], base + 2) * b.wt[k];
    }
    return s;
  }
};

// ------------------------------------------------------------------------
// Surfel providers and Eq. 6.
// ------------------------------------------------------------------------
template <class S> struct Surfel {
  V3<S> mu, tu, tv, a;
  S su, sv, op, m, r;
};

struct SurfelValues {
  const SceneD* sc;
  Surfel<double> get(int i) {
    Surfel<double> s;
    s.mu = sc->mu[i]; s.tu = sc->tu[i]; s.tv = sc->tv[i]; s.a = sc->a[i];
    s.su = sc->su[i]; s.sv = sc->sv[i]; s.op = sc->op[i]; s.m = sc->m[i]; s.r = sc->r[i];
    return s;
  }
};
struct SurfelTape {
  const SceneD* sc;
  std::vector<std::pair<int, int>> inputs;  // (surfel id, tape id of its first parameter)
  Surfel<Var> get(int i) {
    // Parameter order: mu(3) tu(3) tv(3) s_u s_v o a(3) m r  (17 values).
    double p[17] = {sc->mu[i].x, sc->mu[i].y, sc->mu[i].z, sc->tu[i].x, sc->tu[i].y, sc->tu[i].z,
                    sc->tv[i].x, sc->tv[i].y, sc->tv[i].z, sc->su[i], sc->sv[i], sc->op[i],
                    sc->a[i].x, sc->a[i].y, sc->a[i].z, sc->m[i], sc->r[i]};
    Var v[17];
    for (int k = 0; k < 17; ++k) v[k] = make_input(p[k]);
    inputs.push_back({i, v[0].id});
    Surfel<Var> s;
    s.mu = {v[0], v[1], v[2]}; s.tu = {v[3], v[4], v[5]}; s.tv = {v[6], v[7], v[8]};
    s.su = v[9]; s.sv = v[10]; s.op = v[11]; s.a = {v[12], v[13], v[14]}; s.m = v[15]; s.r = v[16];
    return s;
  }
};

// Eq. 6 for one (ray, surfel): plane hit, local coordinates, effective opacity.
template <class S> struct HitS {
  S t, u, v, oG, alpha, denom;
  V3<S> x, n;  // hit position, hit normal facing the ray
};
template <class S> HitS<S> intersect(const Surfel<S>& s, const D3& o, const D3& d, double alpha_max) {
  using std::exp; using std::sqrt;
  HitS<S> h;
  V3<S> c = cross(s.tu, s.tv);
  S cl = sqrt(dot(c, c));
  V3<S> nh = {c.x / cl, c.y / cl, c.z / cl};
  V3<S> dd = lift<S>(d), oo = lift<S>(o);
  h.denom = dot(dd, nh);
  h.t = dot(s.mu - oo, nh) / h.denom;
  h.x = oo + scl(dd, h.t);
  V3<S> q = h.x - s.mu;
  h.u = dot(q, s.tu) / s.su;
  h.v = dot(q, s.tv) / s.sv;
  h.oG = s.op * exp((h.u * h.u + h.v * h.v) * -0.5);
  h.alpha = val(h.oG) > alpha_max ? S(alpha_max) : h.oG;
  h.n = val(h.denom) < 0.0 ? nh : scl(nh, S(-1.0));
  return h;
}

struct Cand { double t; int id; double r2, alpha, oG, g, cosv; };  // g = |grad of r2 / 2| in the plane, cosv = |d.n|

// All candidates of one ray (plane hit in front of the origin); those that
// pass Eq. 6's support and opacity tests are marked accepted.
void collect(const SceneD& sc, const Params& P, const D3& o, const D3& d, std::vector<Cand>& cands,
             std::vector<Cand>& acc) {
  cands.clear(); acc.clear();
  for (int i = 0; i < sc.n; ++i) {
    double denom = dot(d, sc.nh[i]);
    if (std::fabs(denom) < 1e-12) continue;
    double t = dot(sc.mu[i] - o, sc.nh[i]) / denom;
    if (!std::isfinite(t)) continue;
    D3 q = o + scl(d, t) - sc.mu[i];
    double u = dot(q, sc.tu[i]) / sc.su[i], v = dot(q, sc.tv[i]) / sc.sv[i];
    double r2 = u * u + v * v;
    double oG = sc.op[i] * std::exp(-0.5 * r2);
    double alpha = std::min(P.alpha_max, oG);
    const double gu = u / sc.su[i], gv = v / sc.sv[i];
    Cand c{t, i, r2, alpha, oG, std::sqrt(gu * gu + gv * gv), std::fabs(denom)};
    if (r2 <= 4.0 * P.support_r2) cands.push_back(c);  // only near ones can matter for margins
    if (t > P.t_min && r2 <= P.support_r2 && alpha >= P.alpha_min) acc.push_back(c);
  }
  std::sort(acc.begin(), acc.end(), [](const Cand& a, const Cand& b) {
    return a.t < b.t || (a.t == b.t && a.id < b.id);
  });
}

// Ray shift (world units) that moves u^2 + v^2 of a candidate by `dr2`, or
// its alpha~ by `da`: a shift moves the hit point in the plane by up to
// (1 + t) / |cos| of it, and u^2 + v^2 changes by 2 g per unit of that.
double shift_for_r2(const Cand& c, double dr2) {
  return std::fabs(dr2) * c.cosv / (2.0 * std::max(c.g, 1e-300) * (1.0 + std::fabs(c.t)));
}
double shift_for_alpha(const Cand& c, double da) {
  return std::fabs(da) * c.cosv / (std::max(c.alpha * c.g, 1e-300) * (1.0 + std::fabs(c.t)));
}

// Margins of the acceptance decisions of the candidates with t <= t_limit.
// A decision counts only when flipping it could move the result by more than
// IMPACT: accepting or dropping a candidate at the support edge changes its
// weight by T_before * o exp(-R^2/2), at the opacity threshold by
// T_before * alpha_min, where T_before is the transmittance in front of it
// (`prof` holds (t_j, T after hit j) of the composited hits).
const double IMPACT = 1e-5;

double T_before(const std::vector<std::pair<double, double>>* prof, double t) {
  if (!prof) return 1.0;
  double T = 1.0;
  for (const auto& h : *prof) {
    if (h.first < t) T = h.second; else break;
  }
  return T;
}

void candidate_margins(const Params& P, const std::vector<Cand>& cands, const std::vector<double>& op,
                       double t_limit, Margins* mg, const std::vector<std::pair<double, double>>* prof) {
  if (!mg) return;
  for (const Cand& c : cands) {
    if (c.t > t_limit) continue;
    bool in_front = c.t > P.t_min, in_support = c.r2 <= P.support_r2, dense = c.alpha >= P.alpha_min;
    const double Tb = T_before(prof, c.t);
    const double a_edge = op[c.id] * std::exp(-0.5 * P.support_r2);
    // Support edge: matters when the candidate would pass the opacity test there.
    if (in_front && a_edge >= P.alpha_min && Tb * a_edge >= IMPACT) {
      mg->put(M_SUPPORT, (c.r2 - P.support_r2) / P.support_r2);
      mg->put(M_SUPPORT_SHIFT, shift_for_r2(c, c.r2 - P.support_r2));
    }
    if (in_front && in_support && Tb * P.alpha_min >= IMPACT) {
      mg->put(M_ALPHA, (c.alpha - P.alpha_min) / P.alpha_min);
      mg->put(M_ALPHA_SHIFT, shift_for_alpha(c, c.alpha - P.alpha_min));
    }
    if (in_support && dense && Tb * c.alpha >= IMPACT) mg->put(M_TMIN, (c.t - P.t_min) / P.t_min);
  }
}

// Eq. 7 composite of the sorted accepted hits; the stop index is decided on
// the values.  Returns the composited record in scalar type S.
template <class S> struct Record {
  S T, W, depth, m, r, nlen;
  V3<S> x, n, a, rho;
  int hits = 0;
  double t_stop = 0.0;
  int id_stop = -1;
  uint32_t sig = 2166136261u;
};

template <class S, class SP, class EP>
Record<S> composite(SP& surf, EP& env, const Params& P, const D3& o, const D3& d,
                    const std::vector<Cand>& acc, Margins* mg,
                    std::vector<std::pair<double, double>>* prof = nullptr) {
  using std::sqrt;
  Record<S> rec;
  if (prof) prof->clear();
  S T(1.0), W(0.0), St(0.0), Sm(0.0), Sr(0.0);
  V3<S> Sx, Sn, Sa;
  size_t j = 0;
  for (; j < acc.size(); ++j) {
    Surfel<S> s = surf.get(acc[j].id);
    HitS<S> h = intersect(s, o, d, P.alpha_max);
    const double T_in = val(T);  // transmittance in front of hit j
    S w = T * h.alpha;
    W = W + w;
    Sx = Sx + scl(h.x, w);
    St = St + w * h.t;
    Sn = Sn + scl(h.n, w);
    Sa = Sa + scl(s.a, w);
    Sm = Sm + w * s.m;
    Sr = Sr + w * s.r;
    T = T * (1.0 - h.alpha);
    rec.hits++;
    rec.t_stop = acc[j].t;
    rec.id_stop = acc[j].id;
    rec.sig = (rec.sig ^ (uint32_t)acc[j].id) * 16777619u;
    if (prof) prof->push_back({acc[j].t, val(T)});
    if (mg) {
      mg->put(M_STOP, (val(T) - P.T_min) / P.T_min);
      mg->put(M_CAP, val(h.oG) - P.alpha_max);
      // Exactly equal depths (coplanar surfels) are ordered by id on both
      // sides; only distinct but nearly equal depths may swap in FP32.
      // Swapping hits j and j+1 leaves T behind them unchanged and moves the
      // weighted sum of each composited attribute z by exactly
      // T_in alpha_j alpha_j+1 (z_j - z_j+1) (position and depth by the tiny
      // depth gap), the record z / W by that over W >= 1 - T behind both, so
      // a near tie counts only when that change reaches IMPACT.
      double swap = 0.0;
      if (j + 1 < acc.size()) {
        const SceneD& sd = *surf.sc;
        const int i0 = acc[j].id, i1 = acc[j + 1].id;
        const double f0 = dot(d, sd.nh[i0]) < 0.0 ? 1.0 : -1.0, f1 = dot(d, sd.nh[i1]) < 0.0 ? 1.0 : -1.0;
        const D3 dn = scl(sd.nh[i0], f0) - scl(sd.nh[i1], f1), da = sd.a[i0] - sd.a[i1];
        const double dz = std::max({std::fabs(dn.x), std::fabs(dn.y), std::fabs(dn.z), std::fabs(da.x),
                                    std::fabs(da.y), std::fabs(da.z), std::fabs(sd.m[i0] - sd.m[i1]),
                                    std::fabs(sd.r[i0] - sd.r[i1])});
        const double a0 = val(h.alpha), a1 = acc[j + 1].alpha;
        swap = T_in * a0 * a1 * dz / std::max(1e-300, 1.0 - T_in * (1.0 - a0) * (1.0 - a1));
        // when the composite stops at hit j, a swap composites hit j+1 in its place
        if (val(T) < P.T_min) swap = T_in;
      }
      if (j + 1 < acc.size() && acc[j + 1].t != acc[j].t && swap >= IMPACT) {
        const double gap = acc[j + 1].t - acc[j].t;
        mg->put(M_TIE, gap / std::max(1.0, std::fabs(acc[j].t)));
        // t_k = (mu_k - o).n_k / (d.n_k): a shift of the origin moves the gap
        // by the shift times n_j+1 / (d.n_j+1) - n_j / (d.n_j)
        const D3& n0 = surf.sc->nh[acc[j].id];
        const D3& n1 = surf.sc->nh[acc[j + 1].id];
        const D3 dv = scl(n1, 1.0 / dot(d, n1)) - scl(n0, 1.0 / dot(d, n0));
        const double sens = norm(dv) * (1.0 + std::fabs(acc[j].t));
        if (sens > 0.0) mg->put(M_TIE_SHIFT, gap / sens);
      }
    }
    if (val(T) < P.T_min) { ++j; break; }
  }
  S inv = 1.0 / (W + P.eps_w);
  rec.T = T; rec.W = W;
  rec.x = scl(Sx, inv); rec.depth = St * inv; rec.a = scl(Sa, inv); rec.m = Sm * inv; rec.r = Sr * inv;
  V3<S> mv = scl(Sn, inv);
  rec.nlen = sqrt(dot(mv, mv));
  if (val(rec.nlen) < 1e-12) rec.n = lift<S>(scl(d, -1.0));
  else rec.n = scl(mv, 1.0 / rec.nlen);
  V3<S> Ed = env.lookup(d);
  rec.rho = Sa + scl(Ed, T);
  return rec;
}

// Shadow ray: V = prod (1 - alpha~) over all accepted hits, 0 once < T_min.
double shadow(const SceneD& sc, const Params& P, const D3& o, const D3& d, std::vector<Cand>& cands,
              std::vector<Cand>& acc, Margins* mg) {
  collect(sc, P, o, d, cands, acc);
  double V = 1.0;
  for (const Cand& c : acc) V *= (1.0 - c.alpha);
  if (mg) {
    mg->put(M_STOP, (V - P.T_min) / P.T_min);
    for (const Cand& c : cands) {
      bool in_front = c.t > P.t_min, in_support = c.r2 <= P.support_r2, dense = c.alpha >= P.alpha_min;
      const double a_edge = sc.op[c.id] * std::exp(-0.5 * P.support_r2);
      if (in_front && a_edge >= P.alpha_min && V * a_edge >= IMPACT) {
        mg->put(M_SUPPORT, (c.r2 - P.support_r2) / P.support_r2);
        mg->put(M_SUPPORT_SHIFT, shift_for_r2(c, c.r2 - P.support_r2));
      }
      if (in_front && in_support && V * P.alpha_min >= IMPACT) {
        mg->put(M_ALPHA, (c.alpha - P.alpha_min) / P.alpha_min);
        mg->put(M_ALPHA_SHIFT, shift_for_alpha(c, c.alpha - P.alpha_min));
      }
      if (in_support && dense && V * c.alpha >= IMPACT) mg->put(M_TMIN, (c.t - P.t_min) / P.t_min);
    }
  }
  return V < P.T_min ? 0.0 : V;
}

// ------------------------------------------------------------------------
// BRDF (metallic-roughness: Lambert + GGX / Smith / Schlick).
// ------------------------------------------------------------------------
template <class S>
V3<S> brdf(const V3<S>& n, const D3& wo, const D3& wi, const V3<S>& a, const S& m, const S& r, int mode) {
  using std::sqrt;
  V3<S> zero;
  S ci = dot(n, lift<S>(wi)), co = dot(n, lift<S>(wo));
  if (val(ci) <= 0.0 || val(co) <= 0.0) return zero;
  if (mode == 1) return scl(a, 1.0 / PI);
  S one_m = 1.0 - m;
  V3<S> kd = scl(a, one_m);
  V3<S> F0 = {0.04 * one_m + a.x * m, 0.04 * one_m + a.y * m, 0.04 * one_m + a.z * m};
  S ag = r * r;
  S a2 = ag * ag;
  D3 h = normalize(wi + wo);
  S nh = dot(n, lift<S>(h));
  double oh = dot(wo, h);
  S den = nh * nh * (a2 - 1.0) + 1.0;
  S D = a2 / (den * den * PI);
  S G1i = 2.0 * ci / (ci + sqrt(a2 + (1.0 - a2) * ci * ci));
  S G1o = 2.0 * co / (co + sqrt(a2 + (1.0 - a2) * co * co));
  double fw = std::pow(1.0 - oh, 5.0);
  S spec = D * G1i * G1o / (ci * co * 4.0);
  V3<S> F = {F0.x + (1.0 - F0.x) * fw, F0.y + (1.0 - F0.y) * fw, F0.z + (1.0 - F0.z) * fw};
  return {kd.x / PI + F.x * spec, kd.y / PI + F.y * spec, kd.z / PI + F.z * spec};
}

// Orthonormal basis around n (Duff, Burgess, Christensen, Hery, Kensler,
// Liani, Villemin 2017): returns b1, b2 with (b1, b2, n) right-handed.
void onb(const D3& n, D3& b1, D3& b2) {
  double sgn = std::copysign(1.0, n.z);
  double a = -1.0 / (sgn + n.z);
  double b = n.x * n.y * a;
  b1 = {1.0 + sgn * n.x * n.x * a, sgn * b, -sgn * n.x};
  b2 = {b, sgn + n.y * n.y * a, -n.y};
}

double ggx_D(double nh, double a2) {
  double den = nh * nh * (a2 - 1.0) + 1.0;
  return a2 / (PI * den * den);
}

// GGX half-vector sample (Walter et al. 2007, D(h)(n.h) density) mirrored about h.
D3 sample_ggx(const D3& n, const D3& wo, double r, double u1, double u2) {
  double ag = r * r, a2 = ag * ag;
  double c2 = (1.0 - u1) / (1.0 + (a2 - 1.0) * u1);
  double ct = std::sqrt(std::max(0.0, c2)), st = std::sqrt(std::max(0.0, 1.0 - c2));
  double ph = 2.0 * PI * u2;
  D3 b1, b2;
  onb(n, b1, b2);
  D3 h = scl(b1, st * std::cos(ph)) + scl(b2, st * std::sin(ph)) + scl(n, ct);
  double oh = dot(wo, h);
  return scl(h, 2.0 * oh) - wo;
}

// Cosine-weighted hemisphere sample (Malley's method).
D3 sample_cos(const D3& n, double u1, double u2) {
  double rr = std::sqrt(u1), ph = 2.0 * PI * u2;
  D3 b1, b2;
  onb(n, b1, b2);
  return scl(b1, rr * std::cos(ph)) + scl(b2, rr * std::sin(ph)) + scl(n, std::sqrt(std::max(0.0, 1.0 - u1)));
}

double pdf_ggx(const D3& n, const D3& wo, const D3& wi, double r) {
  D3 hs = wi + wo;
  double hl = norm(hs);
  if (hl <= 0.0) return 0.0;
  D3 h = scl(hs, 1.0 / hl);
  double nh = dot(n, h), oh = dot(wo, h);
  if (nh <= 0.0 || oh <= 0.0) return 0.0;
  double ag = r * r;
  return ggx_D(nh, ag * ag) * nh / (4.0 * oh);
}
double pdf_bsdf(const D3& n, const D3& wo, const D3& wi, double r, double p_spec) {
  double pc = std::max(0.0, dot(n, wi)) / PI;
  double pg = p_spec > 0.0 ? pdf_ggx(n, wo, wi, r) : 0.0;
  return p_spec * pg + (1.0 - p_spec) * pc;
}

// ------------------------------------------------------------------------
// Camera rays (pinhole, pixel centres, vertical field of view).
// ------------------------------------------------------------------------
struct Cam { D3 eye, f, r, u; double th, aspect; int W, H; };
Cam make_cam(const double eye[3], const double target[3], const double up[3], double fovy, int W, int H) {
  Cam c;
  c.eye = {eye[0], eye[1], eye[2]};
  c.f = normalize(D3{target[0] - eye[0], target[1] - eye[1], target[2] - eye[2]});
  c.r = normalize(cross(c.f, D3{up[0], up[1], up[2]}));
  c.u = cross(c.r, c.f);
  c.th = std::tan(0.5 * fovy * PI / 180.0);
  c.aspect = (double)W / (double)H;
  c.W = W; c.H = H;
  return c;
}
// The pixel ray is the FP64 pinhole direction rounded once to FP32: the
// renderer's rays are FP32 vectors, and rounding the same FP64 direction on
// both sides makes them trace the same ray.
D3 cam_dir(const Cam& c, int p) {
  int x = p % c.W, y = p / c.W;
  double sx = (((double)x + 0.5) / c.W * 2.0 - 1.0) * c.th * c.aspect;
  double sy = (1.0 - ((double)y + 0.5) / c.H * 2.0) * c.th;
  D3 d = normalize(c.f + scl(c.r, sx) + scl(c.u, sy));
  return {(double)(float)d.x, (double)(float)d.y, (double)(float)d.z};
}

// ------------------------------------------------------------------------
// Eq. 11 per pixel: frozen sample data (directions, pdfs, MIS weights,
// visibilities, secondary records) from the record of theta_0, then the live
// evaluation.
// ------------------------------------------------------------------------
struct SampleFz {
  int e_ok = 0; D3 we; double pe = 0, wenv = 0, Ve = 0;
  int b_ok = 0; D3 wi; double pb = 0, wbsdf = 0, T2 = 1; int sec_ok = 0;
  int q_ok[2] = {0, 0}; D3 wq[2]; double pq[2] = {0, 0}, Vq[2] = {0, 0}; D3 fcos_q[2];
};

struct Work {  // per-thread scratch
  std::vector<Cand> cands, acc;
  std::vector<std::pair<double, double>> prof;
};

// Sample data of one pixel.  Margins: `mg` (nullable) receives every shading
// decision of the pixel; `smg` (nullable) receives one entry per sample with
// that sample's own decisions plus the pixel-level ones (view cosine and
// frame orientation at the primary record), which every sample depends on.
void frozen_samples(const SceneD& sc, const Env& env0, const Params& P, const Record<double>& rec,
                    const D3& d, uint32_t pixel, int spp, uint64_t seed, Work& wk,
                    std::vector<SampleFz>& out, Margins* mg, int64_t* rays, std::vector<Margins>* smg = nullptr) {
  out.assign(spp, SampleFz());
  if (smg) smg->assign(spp, Margins());
  if (rec.hits == 0) return;
  D3 wo = scl(d, -1.0), n = rec.n;
  D3 xs = rec.x + scl(n, P.ray_offset);
  double co = dot(n, wo);
  // View-side cosine (the Lambert term makes the estimator jump at 0) and the
  // sign of n_z that orients the sampling frame (an exact 0 is the same on
  // both sides).
  Margins pix;
  pix.put(M_COS, co);
  if (n.z != 0.0) pix.put(M_FRAME, n.z);
  if (mg) mg->merge(pix);
  if (smg) for (Margins& m : *smg) m.merge(pix);
  if (co <= 0.0) return;
  const double ps = P.brdf_mode == 1 ? 0.0 : P.p_spec;
  SurfelValues sv{&sc};
  EnvValues ev{&env0};
  for (int s = 0; s < spp; ++s) {
    SampleFz& fz = out[s];
    Margins ms;
    Margins* m = (mg || smg) ? &ms : nullptr;
    double u[9];
    sample_uniforms(pixel, (uint32_t)s, seed, P.sampler, u);
    if (P.sampling_mode != 1) {  // (i) environment NEE at the primary record
      env_sample(env0, u[0], u[1], fz.we, fz.pe, m);
      double ce = dot(n, fz.we);
      if (ce > 0.0 && fz.pe > 0.0) {
        fz.e_ok = 1;
        fz.Ve = shadow(sc, P, xs, fz.we, wk.cands, wk.acc, m);
        if (rays) ++*rays;
        double pb = pdf_bsdf(n, wo, fz.we, rec.r, ps);
        fz.wenv = P.sampling_mode == 2 ? 1.0 : fz.pe * fz.pe / (fz.pe * fz.pe + pb * pb);
      }
    }
    // (ii) BSDF continuation from the cosine/GGX mixture
    fz.wi = (u[2] < ps) ? sample_ggx(n, wo, rec.r, u[3], u[4]) : sample_cos(n, u[3], u[4]);
    double ci = dot(n, fz.wi);
    double pb = pdf_bsdf(n, wo, fz.wi, rec.r, ps);
    if (ci > 0.0 && pb > 0.0) {
      fz.b_ok = 1;
      fz.pb = pb;
      if (P.sampling_mode == 1) {
        fz.wbsdf = 1.0;
      } else {
        double pe_i = env_pdf(env0, fz.wi, m);
        fz.wbsdf = pb * pb / (pb * pb + pe_i * pe_i);
      }
      collect(sc, P, xs, fz.wi, wk.cands, wk.acc);
      Record<double> r2 = composite<double>(sv, ev, P, xs, fz.wi, wk.acc, m, &wk.prof);
      candidate_margins(P, wk.cands, sc.op, r2.hits && val(r2.T) < P.T_min ? r2.t_stop : 1e300, m, &wk.prof);
      if (rays) ++*rays;
      fz.T2 = r2.T;
      if (r2.hits > 0) {
        fz.sec_ok = 1;
        D3 n2 = r2.n, wo2 = scl(fz.wi, -1.0);
        D3 xs2 = r2.x + scl(n2, P.ray_offset);
        double co2 = dot(n2, wo2);
        if (m) m->put(M_COS, co2);
        for (int q = 0; q < 2; ++q) {
          env_sample(env0, u[5 + 2 * q], u[6 + 2 * q], fz.wq[q], fz.pq[q], m);
          double cq = dot(n2, fz.wq[q]);
          if (!(cq > 0.0 && co2 > 0.0 && fz.pq[q] > 0.0)) continue;
          fz.q_ok[q] = 1;
          fz.Vq[q] = shadow(sc, P, xs2, fz.wq[q], wk.cands, wk.acc, m);
          if (rays) ++*rays;
          D3 f2 = brdf<double>(n2, wo2, fz.wq[q], r2.a, r2.m, r2.r, P.brdf_mode);
          fz.fcos_q[q] = scl(f2, cq);
        }
      }
    }
    if (mg) mg->merge(ms);
    if (smg) (*smg)[s].merge(ms);
  }
}

// Pixel value L = T E(d) + (1 - T) / S * sum_s c_s, c_s = c_e + c_b of
// Eq. 11.  `per_sample` (nullable, spp entries) receives each term c_s.
template <class S, class EP>
V3<S> eval_pixel(const Record<S>& rec, EP& env, const Params& P, const D3& d, const std::vector<SampleFz>& fzs,
                 int spp, V3<S>* per_sample = nullptr) {
  D3 wo = scl(d, -1.0);
  V3<S> Ld = env.lookup(d);
  V3<S> sum;
  for (int s = 0; s < spp && rec.hits > 0; ++s) {
    const SampleFz& fz = fzs[s];
    V3<S> cs;
    if (fz.e_ok) {
      V3<S> f = brdf<S>(rec.n, wo, fz.we, rec.a, rec.m, rec.r, P.brdf_mode);
      S c = dot(rec.n, lift<S>(fz.we)) * (fz.Ve * fz.wenv / fz.pe);
      V3<S> E = env.lookup(fz.we);
      cs = cs + scl(mul(f, E), c);
    }
    if (fz.b_ok) {
      V3<S> f = brdf<S>(rec.n, wo, fz.wi, rec.a, rec.m, rec.r, P.brdf_mode);
      S c = dot(rec.n, lift<S>(fz.wi)) / fz.pb;
      V3<S> beta = scl(f, c);
      V3<S> inc;
      if (P.sampling_mode != 2) inc = scl(env.lookup(fz.wi), fz.wbsdf * fz.T2);
      if (fz.sec_ok) {
        for (int q = 0; q < 2; ++q) {
          if (!fz.q_ok[q]) continue;
          V3<S> E = env.lookup(fz.wq[q]);
          double k = (1.0 - fz.T2) * 0.5 * fz.Vq[q] / fz.pq[q];
          inc = inc + V3<S>(E.x * (fz.fcos_q[q].x * k), E.y * (fz.fcos_q[q].y * k), E.z * (fz.fcos_q[q].z * k));
        }
      }
      cs = cs + mul(beta, inc);
    }
    sum = sum + cs;
    if (per_sample) per_sample[s] = cs;
  }
  S A = 1.0 - rec.T;
  S kA = A / (double)spp;
  return scl(Ld, rec.T) + scl(sum, kA);
}

// ------------------------------------------------------------------------
// Output layout of one pixel (NCH doubles).
// ------------------------------------------------------------------------
enum {
  CH_T, CH_W, CH_DEPTH, CH_X, CH_N = CH_X + 3, CH_A = CH_N + 3, CH_M = CH_A + 3, CH_R, CH_RHO,
  CH_NLEN = CH_RHO + 3, CH_HITS, CH_TSTOP, CH_IDSTOP, CH_SIG, NCH
};
const int NDIFF = CH_NLEN;  // channels 0..16 carry gradients

template <class S> void record_to_channels(const Record<S>& r, S* ch) {
  ch[CH_T] = r.T; ch[CH_W] = r.W; ch[CH_DEPTH] = r.depth;
  ch[CH_X] = r.x.x; ch[CH_X + 1] = r.x.y; ch[CH_X + 2] = r.x.z;
  ch[CH_N] = r.n.x; ch[CH_N + 1] = r.n.y; ch[CH_N + 2] = r.n.z;
  ch[CH_A] = r.a.x; ch[CH_A + 1] = r.a.y; ch[CH_A + 2] = r.a.z;
  ch[CH_M] = r.m; ch[CH_R] = r.r;
  ch[CH_RHO] = r.rho.x; ch[CH_RHO + 1] = r.rho.y; ch[CH_RHO + 2] = r.rho.z;
}

SceneD load_scene(const float* mu, const float* tu, const float* tv, const float* scale, const float* op,
                  const float* al, const float* me, const float* ro, int n) {
  SceneD s;
  s.n = n;
  s.mu.resize(n); s.tu.resize(n); s.tv.resize(n); s.nh.resize(n); s.a.resize(n);
  s.su.resize(n); s.sv.resize(n); s.op.resize(n); s.m.resize(n); s.r.resize(n);
  for (int i = 0; i < n; ++i) {
    s.mu[i] = {mu[3 * i], mu[3 * i + 1], mu[3 * i + 2]};
    s.tu[i] = {tu[3 * i], tu[3 * i + 1], tu[3 * i + 2]};
    s.tv[i] = {tv[3 * i], tv[3 * i + 1], tv[3 * i + 2]};
    s.nh[i] = normalize(cross(s.tu[i], s.tv[i]));
    s.a[i] = {al[3 * i], al[3 * i + 1], al[3 * i + 2]};
    s.su[i] = scale[2 * i]; s.sv[i] = scale[2 * i + 1];
    s.op[i] = op[i]; s.m[i] = me[i]; s.r[i] = ro[i];
  }
  return s;
}

}  // namespace

// ==========================================================================
// C interface (consumed by oracle/__init__.py through ctypes).
// ==========================================================================
extern "C" {

struct or_scene {
  const float *mu, *tu, *tv, *scale, *opacity, *albedo, *metallic, *roughness;
  int n;
};
struct or_camera { double eye[3], target[3], up[3], fovy_deg; int width, height; };
struct or_params {
  double T_min, alpha_min, alpha_max, support_r2, eps_w, t_min, ray_offset, p_spec;
  int brdf_mode, sampling_mode, sampler;
};

int or_nch() { return NCH; }
int or_nmargin() { return NMARGIN; }

void or_philox(const uint32_t* ctr, int n, uint32_t k0, uint32_t k1, uint32_t* out) {
  for (int i = 0; i < n; ++i) philox4x32_10(ctr + 4 * i, k0, k1, out + 4 * i);
}

void or_uniforms(uint32_t pixel, uint32_t sample, uint64_t seed, int sampler, double* u9) {
  sample_uniforms(pixel, sample, seed, sampler, u9);
}

void or_sobol(const uint32_t* index, int n, int dim, uint32_t* out) {
  for (int i = 0; i < n; ++i) out[i] = sobol32(index[i], dim);
}

static Params to_params(const or_params* p) {
  return Params{p->T_min, p->alpha_min, p->alpha_max, p->support_r2, p->eps_w, p->t_min,
                p->ray_offset, p->p_spec, p->brdf_mode, p->sampling_mode, p->sampler};
}
static SceneD to_scene(const or_scene* s) {
  return load_scene(s->mu, s->tu, s->tv, s->scale, s->opacity, s->albedo, s->metallic, s->roughness, s->n);
}

// Environment tables (FP64) for inspection.
void or_env_tables(const float* rgb, int H, int W, double* pmf_row, double* cdf_row, double* pmf_col,
                   double* cdf_col) {
  Env e; e.H = H; e.W = W; e.rgb = rgb;
  build_env_tables(e);
  std::memcpy(pmf_row, e.pmf_row.data(), sizeof(double) * H);
  std::memcpy(cdf_row, e.cdf_row.data(), sizeof(double) * H);
  std::memcpy(pmf_col, e.pmf_col.data(), sizeof(double) * H * W);
  std::memcpy(cdf_col, e.cdf_col.data(), sizeof(double) * H * W);
}

void or_env_sample(const float* rgb, int H, int W, const double* u, int n, double* dirs, double* pdf) {
  Env e; e.H = H; e.W = W; e.rgb = rgb;
  build_env_tables(e);
  for (int i = 0; i < n; ++i) {
    D3 w;
    env_sample(e, u[2 * i], u[2 * i + 1], w, pdf[i]);
    dirs[3 * i] = w.x; dirs[3 * i + 1] = w.y; dirs[3 * i + 2] = w.z;
  }
}

void or_env_eval(const float* rgb, int H, int W, const double* dirs, int n, double* value, double* pdf) {
  Env e; e.H = H; e.W = W; e.rgb = rgb;
  build_env_tables(e);
  EnvValues ev{&e};
  for (int i = 0; i < n; ++i) {
    D3 w{dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2]};
    V3<double> E = ev.lookup(w);
    value[3 * i] = E.x; value[3 * i + 1] = E.y; value[3 * i + 2] = E.z;
    if (pdf) pdf[i] = env_pdf(e, w);
  }
}

// GGX normal distribution D(n.h) for roughness r (alpha_g = r^2).
double or_ggx_D(double nh, double r) { return ggx_D(nh, r * r * r * r); }

// BRDF value f(wi, wo) for arrays of (n, wo, wi, a, m, r).
void or_brdf(const double* n, const double* wo, const double* wi, const double* a, const double* m,
             const double* r, int count, int mode, double* out) {
  for (int i = 0; i < count; ++i) {
    D3 nn{n[3 * i], n[3 * i + 1], n[3 * i + 2]}, o{wo[3 * i], wo[3 * i + 1], wo[3 * i + 2]},
        w{wi[3 * i], wi[3 * i + 1], wi[3 * i + 2]}, aa{a[3 * i], a[3 * i + 1], a[3 * i + 2]};
    V3<double> f = brdf<double>(nn, o, w, aa, m[i], r[i], mode);
    out[3 * i] = f.x; out[3 * i + 1] = f.y; out[3 * i + 2] = f.z;
  }
}

// BSDF mixture sample and pdf: u = (lobe, u1, u2) per sample.
void or_bsdf_sample(const double* n, const double* wo, double r, double p_spec, const double* u, int count,
                    double* wi, double* pdf) {
  D3 nn{n[0], n[1], n[2]}, o{wo[0], wo[1], wo[2]};
  for (int i = 0; i < count; ++i) {
    D3 w = (u[3 * i] < p_spec) ? sample_ggx(nn, o, r, u[3 * i + 1], u[3 * i + 2])
                               : sample_cos(nn, u[3 * i + 1], u[3 * i + 2]);
    wi[3 * i] = w.x; wi[3 * i + 1] = w.y; wi[3 * i + 2] = w.z;
    pdf[i] = pdf_bsdf(nn, o, w, r, p_spec);
  }
}

void or_bsdf_pdf(const double* n, const double* wo, double r, double p_spec, const double* wi, int count,
                 double* pdf) {
  D3 nn{n[0], n[1], n[2]}, o{wo[0], wo[1], wo[2]};
  for (int i = 0; i < count; ++i) pdf[i] = pdf_bsdf(nn, o, D3{wi[3 * i], wi[3 * i + 1], wi[3 * i + 2]}, r, p_spec);
}

// Explicit rays: Eq. 6-7 composite per ray (channels as in or_render).
void or_trace_rays(const or_scene* sc_in, const float* env_rgb, int H, int W, const or_params* pp,
                   const double* orig, const double* dirs, int n_rays, double* ch_out, double* margins) {
  SceneD sc = to_scene(sc_in);
  Params P = to_params(pp);
  Env e; e.H = H; e.W = W; e.rgb = env_rgb;
  SurfelValues sv{&sc};
  EnvValues ev{&e};
  Work wk;
  for (int i = 0; i < n_rays; ++i) {
    D3 o{orig[3 * i], orig[3 * i + 1], orig[3 * i + 2]}, d{dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2]};
    Margins mg;
    collect(sc, P, o, d, wk.cands, wk.acc);
    Record<double> r = composite<double>(sv, ev, P, o, d, wk.acc, &mg, &wk.prof);
    candidate_margins(P, wk.cands, sc.op, r.hits && r.T < P.T_min ? r.t_stop : 1e300, &mg, &wk.prof);
    double* ch = ch_out + (size_t)i * NCH;
    record_to_channels(r, ch);
    ch[CH_NLEN] = r.nlen; ch[CH_HITS] = r.hits; ch[CH_TSTOP] = r.t_stop; ch[CH_IDSTOP] = r.id_stop;
    ch[CH_SIG] = (double)r.sig;
    if (margins) for (int k = 0; k < NMARGIN; ++k) margins[(size_t)i * NMARGIN + k] = mg.m[k];
  }
}

void or_shadow_rays(const or_scene* sc_in, const or_params* pp, const double* orig, const double* dirs, int n_rays,
                    double* vis) {
  SceneD sc = to_scene(sc_in);
  Params P = to_params(pp);
  Work wk;
  for (int i = 0; i < n_rays; ++i) {
    D3 o{orig[3 * i], orig[3 * i + 1], orig[3 * i + 2]}, d{dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2]};
    vis[i] = shadow(sc, P, o, d, wk.cands, wk.acc, nullptr);
  }
}

// Pixel ray directions (the FP64 pinhole direction rounded once to FP32).
void or_camera_dirs(const or_camera* cam_in, const int* pixels, int n, double* dirs) {
  Cam cam = make_cam(cam_in->eye, cam_in->target, cam_in->up, cam_in->fovy_deg, cam_in->width, cam_in->height);
  for (int i = 0; i < n; ++i) {
    const D3 d = cam_dir(cam, pixels[i]);
    dirs[3 * i] = d.x;
    dirs[3 * i + 1] = d.y;
    dirs[3 * i + 2] = d.z;
  }
}

// Render a set of camera pixels.  `sc0`/`env0` are the parameters the frozen
// sample data come from (path replay); pass the same pointers as `sc`/`env`
// for an ordinary render.  Outputs per pixel: NCH channels, RGB radiance
// (when shade != 0), 2 x NMARGIN margins (nullable): those of the primary
// ray, then those of every shading ray of the pixel.  Per sample (nullable,
// pixel-major, spp entries per pixel): the term c_s of Eq. 11 (RGB) and
// NMARGIN margins of that sample's decisions (with the pixel-level shading
// decisions folded in).  Returns the number of rays traced (primary +
// shadow + continuation).
int64_t or_render(const or_scene* sc_in, const or_scene* sc0_in, const or_camera* cam_in, const float* env_rgb,
                  const float* env0_rgb, int H, int W, const or_params* pp, const int* pixels, int n_pix, int spp,
                  uint64_t seed, int shade, double* ch_out, double* rgb_out, double* margins, int n_threads,
                  double* samp_rgb, double* samp_margins) {
  SceneD sc = to_scene(sc_in);
  SceneD sc0 = (sc0_in && sc0_in != sc_in) ? to_scene(sc0_in) : SceneD();
  const SceneD& base = (sc0_in && sc0_in != sc_in) ? sc0 : sc;
  Params P = to_params(pp);
  Env e; e.H = H; e.W = W; e.rgb = env_rgb;
  Env e0; e0.H = H; e0.W = W; e0.rgb = env0_rgb ? env0_rgb : env_rgb;
  build_env_tables(e0);
  Cam cam = make_cam(cam_in->eye, cam_in->target, cam_in->up, cam_in->fovy_deg, cam_in->width, cam_in->height);
  int64_t total_rays = 0;
  if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel num_threads(n_threads) reduction(+ : total_rays)
  {
    Work wk;
    std::vector<SampleFz> fzs;
    std::vector<Margins> smg;
    std::vector<V3<double>> terms;
    SurfelValues sv{&sc}, sv0{&base};
    EnvValues ev{&e}, ev0{&e0};
#pragma omp for schedule(dynamic, 1)
    for (int i = 0; i < n_pix; ++i) {
      int p = pixels[i];
      D3 d = cam_dir(cam, p);
      Margins mg, mgs;  // primary ray; shading rays
      int64_t rays = 1;
      collect(sc, P, cam.eye, d, wk.cands, wk.acc);
      Record<double> r = composite<double>(sv, ev, P, cam.eye, d, wk.acc, &mg, &wk.prof);
      candidate_margins(P, wk.cands, sc.op, r.hits && r.T < P.T_min ? r.t_stop : 1e300, &mg, &wk.prof);
      double* ch = ch_out + (size_t)i * NCH;
      record_to_channels(r, ch);
      ch[CH_NLEN] = r.nlen; ch[CH_HITS] = r.hits; ch[CH_TSTOP] = r.t_stop; ch[CH_IDSTOP] = r.id_stop;
      ch[CH_SIG] = (double)r.sig;
      if (shade) {
        Record<double> r0 = r;
        if (&base != &sc) {
          collect(base, P, cam.eye, d, wk.cands, wk.acc);
          r0 = composite<double>(sv0, ev0, P, cam.eye, d, wk.acc, nullptr);
        }
        frozen_samples(base, e0, P, r0, d, (uint32_t)p, spp, seed, wk, fzs, &mgs, &rays,
                       samp_margins ? &smg : nullptr);
        terms.assign(spp, V3<double>());
        V3<double> L = eval_pixel<double>(r, ev, P, d, fzs, spp, terms.data());
        rgb_out[3 * i] = L.x; rgb_out[3 * i + 1] = L.y; rgb_out[3 * i + 2] = L.z;
        for (int s = 0; s < spp; ++s) {
          const size_t o = (size_t)i * spp + s;
          if (samp_rgb) { samp_rgb[3 * o] = terms[s].x; samp_rgb[3 * o + 1] = terms[s].y; samp_rgb[3 * o + 2] = terms[s].z; }
          if (samp_margins) for (int k = 0; k < NMARGIN; ++k) samp_margins[o * NMARGIN + k] = smg[s].m[k];
        }
      }
      if (margins)
        for (int k = 0; k < NMARGIN; ++k) {
          margins[(size_t)i * 2 * NMARGIN + k] = mg.m[k];
          margins[(size_t)i * 2 * NMARGIN + NMARGIN + k] = mgs.m[k];
        }
      total_rays += rays;
    }
  }
  return total_rays;
}

// Gradient of  sum_i dL_drgb[i] . rgb[i] + sum_i dL_dch[i] . ch[i][0..16]
// with respect to the 17 surfel parameters (mu 3, tu 3, tv 3, s 2, o, a 3, m, r)
// and the environment texels, with the sample data frozen at the current
// parameters (path replay).  Gradients are ADDED to d_surfel (N x 17) and
// d_env (H x W x 3); the sum runs in pixel order (deterministic).
void or_grad(const or_scene* sc_in, const or_camera* cam_in, const float* env_rgb, int H, int W,
             const or_params* pp, const int* pixels, int n_pix, int spp, uint64_t seed, int shade,
             const double* dL_drgb, const double* dL_dch, double* d_surfel, double* d_env, int n_threads) {
  SceneD sc = to_scene(sc_in);
  Params P = to_params(pp);
  Env e; e.H = H; e.W = W; e.rgb = env_rgb;
  build_env_tables(e);
  Cam cam = make_cam(cam_in->eye, cam_in->target, cam_in->up, cam_in->fovy_deg, cam_in->width, cam_in->height);
  struct Contrib { std::vector<std::pair<int, double>> surf, env; };
  std::vector<Contrib> per_pixel(n_pix);
  if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel num_threads(n_threads)
  {
    Work wk;
    std::vector<SampleFz> fzs;
    SurfelValues sv{&sc};
    EnvValues ev{&e};
    Tape tape;
    g_tape = &tape;
#pragma omp for schedule(dynamic, 1)
    for (int i = 0; i < n_pix; ++i) {
      int p = pixels[i];
      D3 d = cam_dir(cam, p);
      tape.nodes.clear();
      collect(sc, P, cam.eye, d, wk.cands, wk.acc);
      Record<double> r0 = composite<double>(sv, ev, P, cam.eye, d, wk.acc, nullptr);
      SurfelTape st{&sc, {}};
      EnvTape et{&e, {}};
      Record<Var> r = composite<Var>(st, et, P, cam.eye, d, wk.acc, nullptr);
      Var ch[NDIFF];
      record_to_channels(r, ch);
      Var out[3];
      if (shade) {
        frozen_samples(sc, e, P, r0, d, (uint32_t)p, spp, seed, wk, fzs, nullptr, nullptr);
        V3<Var> L = eval_pixel<Var>(r, et, P, d, fzs, spp);
        out[0] = L.x; out[1] = L.y; out[2] = L.z;
      }
      std::vector<double> adj(tape.nodes.size(), 0.0);
      auto seed_adj = [&](const Var& v, double g) { if (v.id >= 0 && g != 0.0) adj[v.id] += g; };
      if (shade && dL_drgb) for (int c = 0; c < 3; ++c) seed_adj(out[c], dL_drgb[3 * (size_t)i + c]);
      if (dL_dch) for (int c = 0; c < NDIFF; ++c) seed_adj(ch[c], dL_dch[(size_t)i * NDIFF + c]);
      for (int k = (int)tape.nodes.size() - 1; k >= 0; --k) {
        double g = adj[k];
        if (g == 0.0) continue;
        const TNode& nd = tape.nodes[k];
        if (nd.a >= 0) adj[nd.a] += nd.da * g;
        if (nd.b >= 0) adj[nd.b] += nd.db * g;
      }
      Contrib& cb = per_pixel[i];
      for (auto& in : st.inputs)
        for (int k = 0; k < 17; ++k) cb.surf.push_back({in.first * 17 + k, adj[in.second + k]});
      for (auto& kv : et.texel_var)
        for (int k = 0; k < 3; ++k) cb.env.push_back({kv.first * 3 + k, adj[kv.second + k]});
    }
    g_tape = nullptr;
  }
  for (int i = 0; i < n_pix; ++i) {
    for (auto& c : per_pixel[i].surf) d_surfel[c.first] += c.second;
    std::sort(per_pixel[i].env.begin(), per_pixel[i].env.end());
    for (auto& c : per_pixel[i].env) d_env[c.first] += c.second;
  }
}

}  // extern "C"
