// Cooperative traversal of the wide BVH: WIDE consecutive lanes of a warp
// trace one ray together (sm_103a).
//
// At a wide node lane c tests child slot c (the node's two quad planes make
// each of its two loads one contiguous WIDE * 16 B read), the group continues with the nearest
// child it enters and pushes the others on the ray's stack in shared memory;
// at a leaf lane c tests surfel first + c.  Every branch below is uniform over
// the group, so the lanes of a ray never diverge from one another and a warp
// holds 32 / WIDE rays.  Stack entries carry the entry distance of their box:
// an entry beyond the visitor's current far bound is dropped when popped.
#pragma once
#include "lf_common.cuh"

namespace lf {

constexpr int CSTACK = LF_STACK_DEPTH;  // stack entries per ray (a node visit pushes at most WIDE - 1)
static_assert(WIDE == 8 || WIDE == 16 || WIDE == 32, "WIDE must be 8, 16 or 32");

// The lanes of one ray.
struct Grp {
  unsigned mask;  // warp lanes of the group
  int shift;      // first warp lane of the group
  int c;          // lane within the group
};

__device__ __forceinline__ Grp make_grp() {
  Grp g;
  g.c = threadIdx.x & (WIDE - 1);
  g.shift = (threadIdx.x & 31) & ~(WIDE - 1);
  g.mask = WIDE == 32 ? 0xffffffffu : (((1u << WIDE) - 1u) << g.shift);
  return g;
}

// Group-local ballot: bit c set when lane c's predicate holds.
__device__ __forceinline__ unsigned gballot(const Grp& g, bool p) {
  const unsigned b = __ballot_sync(g.mask, p);
  return WIDE == 32 ? b : (b >> g.shift) & ((1u << WIDE) - 1u);
}
template <class T>
__device__ __forceinline__ T gshfl(const Grp& g, T v, int src) {
  return __shfl_sync(g.mask, v, src, WIDE);
}

// Per-ray shared memory: the ray, the traversal stack (parallel arrays), the
// k-buffers' merge scratch and the candidate queue (WIDE entries each).
struct CStack {
  float4* ray;  // the ray (RAY_QUADS quads, make_ray)
  int* code;
  int* cnt;
  float* t;
  unsigned long long* mk;
  int* mc;
  float* ma;
  int* qc;  // candidates waiting for the precise hit test (instance << 24 | record)
};

// Candidates of the quick hit test wait in a per-ray queue and take the
// precise (double-float) test together once LF_DEFER of them are queued (or
// the traversal ends), so one pass of that test serves up to WIDE of them
// instead of the few of one leaf; 0 tests each leaf's candidates at once.
// The k-buffer's far bound is lowered only when the queue is tested, so a
// larger queue culls later.  Measured on the 800x800x16 room step: 20 is the
// fastest (16: +0.3 %, 12: +1.6 %, 24: +0.4 %; 0 made continuation rays 6 %
// slower).
#ifndef LF_DEFER
#define LF_DEFER 20
#endif
static_assert(LF_DEFER >= 0 && LF_DEFER <= WIDE, "the queue holds at most WIDE candidates");

// Bytes of shared memory per ray.
constexpr int CRAY_SMEM = RAY_QUADS * 16 + CSTACK * (2 * (int)sizeof(int) + (int)sizeof(float)) +
                          WIDE * ((int)sizeof(unsigned long long) + (int)sizeof(int) + (int)sizeof(float)) +
                          WIDE * (int)sizeof(int);

// Carves ray `gid`'s arrays out of a block's shared memory holding n_rays rays.
__device__ __forceinline__ CStack ray_smem(unsigned char* smem, int n_rays, int gid) {
  CStack st;
  st.ray = reinterpret_cast<float4*>(smem) + gid * RAY_QUADS;
  unsigned long long* mk = reinterpret_cast<unsigned long long*>(smem + n_rays * RAY_QUADS * 16);
  st.mk = mk + gid * WIDE;
  int* ints = reinterpret_cast<int*>(mk + n_rays * WIDE);
  st.code = ints + gid * CSTACK;
  st.cnt = ints + n_rays * CSTACK + gid * CSTACK;
  st.mc = ints + 2 * n_rays * CSTACK + gid * WIDE;
  float* fl = reinterpret_cast<float*>(ints + 2 * n_rays * CSTACK + n_rays * WIDE);
  st.t = fl + gid * CSTACK;
  st.ma = fl + n_rays * CSTACK + gid * WIDE;
  st.qc = reinterpret_cast<int*>(fl + n_rays * CSTACK + n_rays * WIDE) + gid * WIDE;
  return st;
}

// Appends this lane's candidate `code` (when `cand`) to the ray's queue of
// `qn` entries.  Group-uniform call.
__device__ __forceinline__ void queue_candidates(const Grp& g, int* qc, int& qn, bool cand, int code) {
  const unsigned m = gballot(g, cand);
  if (cand) qc[qn + __popc(m & ((1u << g.c) - 1u))] = code;
  qn += __popc(m);
  __syncwarp(g.mask);
}

// Stack entries name (instance, wide node or leaf) as in the binary
// traversal: instance << 25 | leaf flag (bit 24) | index; the leaf's surfel
// count sits in the parallel `cnt` array.
__device__ __forceinline__ int wentry(int ii, int code) {
  return code >= 0 ? ((ii << 25) | code) : ((ii << 25) | LEAF_BIT | ~code);
}

// Visitor interface (all members group-uniform except inside leaf()):
//   tlo(), thi()  culling interval of the ray
//   leaf(g, ray, ii, first, count, I)  lanes c < count handle surfel first + c
//   done(), abort()
//   finish()      called once when the walk has ended (not after done() or
//                 abort()): tests what the visitor still holds back
//   any_order  true when the result does not depend on the visiting order
//              (shadow rays): the walk then descends into the first hit
//              child slot instead of the nearest one, saving the min-reduce
//              of every node visit
template <class V, class Ray, class Cnt>
__device__ __forceinline__ void coop_traverse(const Grp& g, const Inst* insts, int n_inst, const Ray& ray, V& vis,
                                              const CStack& st, int* status, Cnt& cnt) {
  int sp = 0;
  // a tree of n leaves has fewer than n wide nodes; the budget only guards
  // against a malformed tree
  int budget = 8;
  // instance boxes, WIDE at a time; instance 0 (background) ends up deepest
  for (int i0 = 0; i0 < n_inst; i0 += WIDE) {
    const int ii = i0 + g.c;
    bool hit = false;
    float tn = 0.0f;
    int code = 0, count = 0, nl = 0;
    if (ii < n_inst) {
      const Inst& I = insts[ii];
      nl = I.n_leaves;
      if (I.wroot != INT_MIN &&
          slab(I.lo[0], I.lo[1], I.lo[2], I.hi[0], I.hi[1], I.hi[2], ray, vis.tlo(), vis.thi(), tn)) {
        hit = true;
        code = wentry(ii, I.wroot);
        count = I.wroot_count;
      }
    }
    const unsigned m = gballot(g, hit);
    if (sp + __popc(m) > CSTACK) {
      if (g.c == 0) report(status, LF_ERR_STACK);
      vis.abort();
      return;
    }
    if (hit) {
      const int pos = sp + __popc(m & ((1u << g.c) - 1u));
      st.code[pos] = code;
      st.cnt[pos] = count;
      st.t[pos] = tn;
    }
    sp += __popc(m);
    budget += __reduce_add_sync(g.mask, nl);
  }
  __syncwarp(g.mask);
  while (sp > 0) {
    --sp;
    const float t0 = st.t[sp];
    if (t0 > vis.thi()) continue;
    int e = st.code[sp], ec = st.cnt[sp];
    while (true) {
      const int ii = e >> 25;
      const Inst& I = insts[ii];
      if (e & LEAF_BIT) {
        if (!LF_IN_BOUNDS((e & 0xffffff) + ec - 1, I.n_leaves, status, "leaf surfel") ||
            !LF_IN_BOUNDS(e & 0xffffff, I.n_leaves, status, "leaf first surfel")) {
          vis.abort();
          return;
        }
        if (g.c == 0) cnt.test(ec);
        vis.leaf(g, ray, ii, e & 0xffffff, ec, I);
        if (vis.done()) return;
        break;
      }
      if (--budget < 0) {
        if (g.c == 0) report(status, LF_ERR_STACK);
        vis.abort();
        return;
      }
      if (g.c == 0) cnt.node();
      if (!LF_IN_BOUNDS(e & 0xffffff, I.n_wide, status, "wide node")) {
        vis.abort();
        return;
      }
      const float4* node = I.wnodes + WNODE_Q * (size_t)(e & 0xffffff);
#if LF_WIDE_FP16
      const float4 H = __ldg(node);
      const uint4 S = __ldg(reinterpret_cast<const uint4*>(node + 1 + g.c));
      int code = (int)S.w, count = 0;
      if (code < 0) {  // leaf: count and first surfel from the slot word
        count = ((code >> 24) & 31) + 1;
        code = ~(code & 0xffffff);
      }
      float tn = 0.0f;
      const bool hit = S.w != WSLOT_EMPTY && slab_rel(S, H, ray, vis.tlo(), vis.thi(), tn);
#else
      const float4 A = __ldg(node + g.c), Bx = __ldg(node + WIDE + g.c);
      const int code = __float_as_int(A.w), count = __float_as_int(Bx.w);
      float tn = 0.0f;
      const bool hit = code != INT_MIN && slab(A.x, A.y, A.z, Bx.x, Bx.y, Bx.z, ray, vis.tlo(), vis.thi(), tn);
#endif
      const unsigned m = gballot(g, hit);
      if (m == 0u) break;
      // nearest child: smallest entry distance (positive floats order as their bits)
      int near;
      if (V::any_order) {
        near = __ffs(m) - 1;
      } else {
        const unsigned key = hit ? __float_as_uint(tn) : 0xffffffffu;
        const unsigned kmin = __reduce_min_sync(g.mask, key);
        near = __ffs(gballot(g, hit && key == kmin)) - 1;
      }
      const unsigned others = m & ~(1u << near);
      if (sp + __popc(others) > CSTACK) {
        if (g.c == 0) report(status, LF_ERR_STACK);
        vis.abort();
        return;
      }
      const int mine = wentry(ii, code);
      if (hit && g.c != near) {
        const int pos = sp + __popc(others & ((1u << g.c) - 1u));
        st.code[pos] = mine;
        st.cnt[pos] = count;
        st.t[pos] = tn;
      }
      sp += __popc(others);
      e = gshfl(g, mine, near);
      ec = gshfl(g, count, near);
      __syncwarp(g.mask);
    }
  }
  vis.finish(g, ray);
}

// Shadow ray (cooperative): V = prod(1 - alpha~) over all accepted hits; 0
// once below T_min.  The product of a leaf's factors is formed over the
// group by a butterfly, which leaves every lane with the same bits.
struct ShadowCoop {
  static constexpr bool any_order = true;
  float V;
  bool stop;
  DevParams P;
  const Inst* insts;
  int* qc;
  int qn;
  __device__ __forceinline__ float tlo() const { return P.t_min; }
  __device__ __forceinline__ float thi() const { return BIG_F; }
  __device__ __forceinline__ bool done() const { return stop; }
  __device__ __forceinline__ void abort() { stop = true; }
  __device__ __forceinline__ void absorb(const Grp& g, float f) {
#pragma unroll
    for (int off = WIDE / 2; off > 0; off >>= 1) f *= __shfl_xor_sync(g.mask, f, off, WIDE);
    V *= f;
    if (V < P.T_min) {
      V = 0.0f;
      stop = true;
    }
  }
#if LF_DEFER > 0
  template <class Ray>
  __device__ __forceinline__ void flush(const Grp& g, const Ray& ray) {
    float f = 1.0f;
    if (g.c < qn) {
      const int code = qc[g.c];
      const Inst& I = insts[code >> 24];
      const int l = code & 0xffffff;
      Rec r;
      load_rec3(I.geo, I.n_leaves, l, r);
      load_rec_tail(I.geo, I.n_leaves, l, r);
      float t, tl, alpha;
      if (hit_precise(r, ray.o(), ray.olo(), ray.d(), P, t, tl, alpha)) f = 1.0f - alpha;
    }
    qn = 0;
    __syncwarp(g.mask);
    absorb(g, f);
  }
  template <class Ray>
  __device__ __forceinline__ void leaf(const Grp& g, const Ray& ray, int ii, int first, int count, const Inst& I) {
    bool cand = false;
    if (g.c < count) {
      Rec r;
      load_rec3(I.geo, I.n_leaves, first + g.c, r);
      float t32;
      cand = hit_quick(r, ray.o(), ray.d(), P, t32);
    }
    const int nm = __popc(gballot(g, cand));
    if (nm == 0) return;
    if (qn + nm > WIDE) {
      flush(g, ray);
      if (stop) return;
    }
    queue_candidates(g, qc, qn, cand, (ii << 24) | (first + g.c));
    if (qn >= LF_DEFER) flush(g, ray);
  }
  template <class Ray>
  __device__ __forceinline__ void finish(const Grp& g, const Ray& ray) {
    if (qn > 0) flush(g, ray);
  }
#else
  template <class Ray>
  __device__ __forceinline__ void leaf(const Grp& g, const Ray& ray, int, int first, int count, const Inst& I) {
    float f = 1.0f;
    if (g.c < count) {
      Rec r;
      float t32, t, tl, alpha;
      if (hit_surfel(I.geo, I.n_leaves, first + g.c, ray.o(), ray.olo(), ray.d(), P, r, t32, t, tl, alpha)) f = 1.0f - alpha;
    }
    absorb(g, f);
  }
  template <class Ray>
  __device__ __forceinline__ void finish(const Grp&, const Ray&) {}
#endif
};

// Cooperative k-buffer (K = WIDE): the K smallest hit keys strictly greater
// than the last round's, sorted over the lanes (lane c holds entry c with its
// opacity alpha~).  The accepted candidates of a queue flush are merged in
// one step: every element's place in the merged order is its own index plus
// the number of smaller elements of the other list (counted with ballots,
// two candidates per pass), elements are scattered to those places in
// shared memory and read back; places beyond K fall off.
//
// Transmittance cut: with T the transmittance in front of the round, the
// composite of the sorted buffer stops at the first entry s with
// T prod_{i <= s} (1 - alpha_i) < T_min.  Hits found later can only enter
// in front of s, which moves the stop forward, so nothing beyond entry s is
// ever composited and the far bound of the traversal drops to its depth.
struct NearKCoop {
  static constexpr bool any_order = false;
  unsigned long long bk;    // this lane's entry (~0: empty)
  int bc;                   // its hit code: instance << 24 | leaf
  float ba;                 // its alpha~
  int cnt;                  // entries held
  unsigned long long last;  // keys must exceed this
  unsigned long long kmax;  // largest held key once full
  float Tin;                // transmittance in front of this round's hits
  float tcut;               // far bound: the stop entry's depth, else kmax's once full, else BIG_F
  DevParams P;
  unsigned long long* mk;   // merge scratch in shared memory (WIDE entries per ray)
  int* mc;
  float* ma;

  __device__ __forceinline__ void reset(unsigned long long lk, float T) {
    bk = ~0ull;
    bc = 0;
    ba = 0.0f;
    cnt = 0;
    last = lk;
    kmax = ~0ull;
    Tin = T;
    tcut = BIG_F;
    qn = 0;
  }
  __device__ __forceinline__ float tlo() const { return fmaxf(P.t_min, key_t(last)); }
  __device__ __forceinline__ float thi() const { return tcut; }
  // quick-test window: beyond the far bound, or in front of the last round's
  // largest key (later rounds re-walk the same leaves), with the margins of
  // the quick test, no candidate can enter
  __device__ __forceinline__ bool in_window(float t32) const {
    return !(t32 > tcut * 1.0001f + 1e-6f) && !(t32 < key_t(last) * 0.9999f - 1e-6f);
  }
  __device__ __forceinline__ bool done() const { return false; }
  __device__ __forceinline__ void abort() {
    cnt = 0;
    qn = 0;
  }
  // Merges this lane's candidate (key, hit code, alpha~) into the sorted
  // buffer when `valid`, then lowers the far bound (group-uniform call).
  __device__ __forceinline__ void merge(const Grp& g, bool valid, unsigned long long key, int code, float alpha) {
    const unsigned m = gballot(g, valid);
    if (m == 0u) return;
    int bshift = 0, cshift = 0, rb = 0;
    // Keys are distinct (the surfel id is part of them), so bk > kj is the
    // complement of this lane's bit of the ballot bk < kj.  Two candidates
    // per pass keep two shuffles in flight (continuation rays 1.3 % faster
    // than one per pass).
    unsigned mm = m;
    while (mm) {
      const int j0 = __ffs(mm) - 1;
      mm &= mm - 1u;
      const int j1 = mm ? __ffs(mm) - 1 : j0;
      const bool two = mm != 0u;
      mm &= mm - 1u;
      const unsigned long long k0 = gshfl(g, key, j0), k1 = gshfl(g, key, j1);
      const unsigned b0 = gballot(g, bk < k0), b1 = gballot(g, bk < k1);
      if (g.c == j0) rb = __popc(b0);
      if (two && g.c == j1) rb = __popc(b1);
      bshift += (int)(((b0 >> g.c) & 1u) ^ 1u) + (two ? (int)(((b1 >> g.c) & 1u) ^ 1u) : 0);
      cshift += ((valid && key > k0) ? 1 : 0) + ((two && valid && key > k1) ? 1 : 0);
    }
    const int db = g.c + bshift, dc = rb + cshift;
    if (db < WIDE) {
      mk[db] = bk;
      mc[db] = bc;
      ma[db] = ba;
    }
    if (valid && dc < WIDE) {
      mk[dc] = key;
      mc[dc] = code;
      ma[dc] = alpha;
    }
    __syncwarp(g.mask);
    bk = mk[g.c];
    bc = mc[g.c];
    ba = ma[g.c];
    __syncwarp(g.mask);
    cnt = min(cnt + __popc(m), WIDE);
    if (cnt >= WIDE) kmax = gshfl(g, bk, WIDE - 1);
    // transmittance cut over the sorted buffer
    float q = g.c < cnt ? 1.0f - ba : 1.0f;
#pragma unroll
    for (int off = 1; off < WIDE; off <<= 1) {
      const float v = __shfl_up_sync(g.mask, q, off, WIDE);
      if (g.c >= off) q *= v;
    }
    const unsigned stop = gballot(g, g.c < cnt && Tin * q < P.T_min);
    if (stop) tcut = key_t(gshfl(g, bk, __ffs(stop) - 1));
    else if (cnt >= WIDE) tcut = key_t(kmax);
  }
  // Precise test of record l of instance ii (its first three quads in r).
  template <class Ray>
  __device__ __forceinline__ bool precise(const Ray& ray, const Inst& I, int ii, int l, Rec& r,
                                          unsigned long long& key, int& code, float& alpha) const {
    float t, tl;
    load_rec_tail(I.geo, I.n_leaves, l, r);
    if (!hit_precise(r, ray.o(), ray.olo(), ray.d(), P, t, tl, alpha)) return false;
    key = hit_key(t, tl, rec_id(r));
    code = (ii << 24) | l;
    return key > last && (cnt < WIDE || key < kmax);
  }
  const Inst* insts;
  int* qc;  // candidate queue (LF_DEFER > 0)
  int qn;
#if LF_DEFER > 0
  template <class Ray>
  __device__ __forceinline__ void flush(const Grp& g, const Ray& ray) {
    bool valid = false;
    unsigned long long key = 0ull;
    int code = 0;
    float alpha = 0.0f;
    if (g.c < qn) {
      const int qcode = qc[g.c];
      const int ii = qcode >> 24, l = qcode & 0xffffff;
      const Inst& I = insts[ii];
      Rec r;
      load_rec3(I.geo, I.n_leaves, l, r);
      valid = precise(ray, I, ii, l, r, key, code, alpha);
    }
    qn = 0;
    __syncwarp(g.mask);
    merge(g, valid, key, code, alpha);
  }
  template <class Ray>
  __device__ __forceinline__ void leaf(const Grp& g, const Ray& ray, int ii, int first, int count, const Inst& I) {
    bool cand = false;
    if (g.c < count) {
      Rec r;
      load_rec3(I.geo, I.n_leaves, first + g.c, r);
      float t32;
      cand = hit_quick(r, ray.o(), ray.d(), P, t32) && in_window(t32);
    }
    const int nm = __popc(gballot(g, cand));
    if (nm == 0) return;
    if (qn + nm > WIDE) flush(g, ray);
    queue_candidates(g, qc, qn, cand, (ii << 24) | (first + g.c));
    if (qn >= LF_DEFER) flush(g, ray);
  }
  template <class Ray>
  __device__ __forceinline__ void finish(const Grp& g, const Ray& ray) {
    if (qn > 0) flush(g, ray);
  }
#else
  template <class Ray>
  __device__ __forceinline__ void leaf(const Grp& g, const Ray& ray, int ii, int first, int count, const Inst& I) {
    bool valid = false;
    unsigned long long key = 0ull;
    int code = 0;
    float alpha = 0.0f;
    if (g.c < count) {
      const int l = first + g.c;
      Rec r;
      load_rec3(I.geo, I.n_leaves, l, r);
      float t32;
      if (hit_quick(r, ray.o(), ray.d(), P, t32) && in_window(t32))
        valid = precise(ray, I, ii, l, r, key, code, alpha);
    }
    merge(g, valid, key, code, alpha);
  }
  template <class Ray>
  __device__ __forceinline__ void finish(const Grp&, const Ray&) {}
#endif
};

// Cooperative far k-buffer for the back-to-front adjoint: the K largest hit
// keys below a bound (inclusive on the first round), sorted descending over
// the lanes (lane c holds entry c; 0 = empty).
struct FarKCoop {
  static constexpr bool any_order = false;
  unsigned long long bk;
  int bc;
  int cnt;
  unsigned long long bound;
  bool inclusive;
  unsigned long long kmin;  // smallest held key once full
  float ktl;                // key_t(kmin) once full, else t_min
  DevParams P;
  unsigned long long* mk;   // merge scratch in shared memory (WIDE entries per ray)
  int* mc;

  __device__ __forceinline__ void reset(unsigned long long b, bool incl) {
    bk = 0ull;
    bc = 0;
    cnt = 0;
    bound = b;
    inclusive = incl;
    kmin = 0ull;
    ktl = P.t_min;
    qn = 0;
  }
  __device__ __forceinline__ float tlo() const { return ktl; }
  __device__ __forceinline__ float thi() const { return key_t(bound); }
  __device__ __forceinline__ bool done() const { return false; }
  __device__ __forceinline__ void abort() {
    cnt = 0;
    qn = 0;
  }
  // Precise test of record l of instance ii (its first three quads in r).
  template <class Ray>
  __device__ __forceinline__ bool precise(const Ray& ray, const Inst& I, int ii, int l, Rec& r,
                                          unsigned long long& key, int& code) const {
    float t, tl, alpha;
    load_rec_tail(I.geo, I.n_leaves, l, r);
    if (!hit_precise(r, ray.o(), ray.olo(), ray.d(), P, t, tl, alpha)) return false;
    key = hit_key(t, tl, rec_id(r));
    code = (ii << 24) | l;
    return (key < bound || (key == bound && inclusive)) && (cnt < WIDE || key > kmin);
  }
  // quick-test window: beyond the bound or, once full, in front of kmin's
  // depth (with the margins of the quick test) no candidate can enter
  __device__ __forceinline__ bool in_window(float t32) const {
    return !(t32 > thi() * 1.0001f + 1e-6f) && !(cnt >= WIDE && t32 < ktl * 0.9999f - 1e-6f);
  }
  const Inst* insts;
  int* qc;  // candidate queue (LF_DEFER > 0)
  int qn;
#if LF_DEFER > 0
  template <class Ray>
  __device__ __forceinline__ void flush(const Grp& g, const Ray& ray) {
    bool valid = false;
    unsigned long long key = 0ull;
    int code = 0;
    if (g.c < qn) {
      const int qcode = qc[g.c];
      const int ii = qcode >> 24, l = qcode & 0xffffff;
      const Inst& I = insts[ii];
      Rec r;
      load_rec3(I.geo, I.n_leaves, l, r);
      valid = precise(ray, I, ii, l, r, key, code);
    }
    qn = 0;
    __syncwarp(g.mask);
    merge(g, valid, key, code);
  }
  template <class Ray>
  __device__ __forceinline__ void leaf(const Grp& g, const Ray& ray, int ii, int first, int count, const Inst& I) {
    bool cand = false;
    if (g.c < count) {
      Rec r;
      load_rec3(I.geo, I.n_leaves, first + g.c, r);
      float t32;
      cand = hit_quick(r, ray.o(), ray.d(), P, t32) && in_window(t32);
    }
    const int nm = __popc(gballot(g, cand));
    if (nm == 0) return;
    if (qn + nm > WIDE) flush(g, ray);
    queue_candidates(g, qc, qn, cand, (ii << 24) | (first + g.c));
    if (qn >= LF_DEFER) flush(g, ray);
  }
  template <class Ray>
  __device__ __forceinline__ void finish(const Grp& g, const Ray& ray) {
    if (qn > 0) flush(g, ray);
  }
#else
  template <class Ray>
  __device__ __forceinline__ void finish(const Grp&, const Ray&) {}
  template <class Ray>
  __device__ __forceinline__ void leaf(const Grp& g, const Ray& ray, int ii, int first, int count, const Inst& I) {
    bool valid = false;
    unsigned long long key = 0ull;
    int code = 0;
    if (g.c < count) {
      const int l = first + g.c;
      Rec r;
      load_rec3(I.geo, I.n_leaves, l, r);
      float t32;
      if (hit_quick(r, ray.o(), ray.d(), P, t32) && in_window(t32)) valid = precise(ray, I, ii, l, r, key, code);
    }
    merge(g, valid, key, code);
  }
#endif
  // The leaf's accepted hits merged into the descending buffer in one step,
  // as NearKCoop::merge does it ascending: each element's place is its own
  // index plus the number of larger elements of the other list (keys are
  // distinct, so bk < kj is the complement of this lane's bit of the ballot
  // bk > kj; two candidates per pass), scattered through shared memory;
  // places beyond K fall off.  The buffer ends as the K largest keys of
  // both, in order -- what inserting the candidates one by one gave.
  __device__ __forceinline__ void merge(const Grp& g, bool valid, unsigned long long key, int code) {
    const unsigned m = gballot(g, valid);
    if (m == 0u) return;
    int bshift = 0, cshift = 0, rb = 0;
    unsigned mm = m;
    while (mm) {
      const int j0 = __ffs(mm) - 1;
      mm &= mm - 1u;
      const int j1 = mm ? __ffs(mm) - 1 : j0;
      const bool two = mm != 0u;
      mm &= mm - 1u;
      const unsigned long long k0 = gshfl(g, key, j0), k1 = gshfl(g, key, j1);
      const unsigned b0 = gballot(g, bk > k0), b1 = gballot(g, bk > k1);
      if (g.c == j0) rb = __popc(b0);
      if (two && g.c == j1) rb = __popc(b1);
      bshift += (int)(((b0 >> g.c) & 1u) ^ 1u) + (two ? (int)(((b1 >> g.c) & 1u) ^ 1u) : 0);
      cshift += ((valid && key < k0) ? 1 : 0) + ((two && valid && key < k1) ? 1 : 0);
    }
    const int db = g.c + bshift, dc = rb + cshift;
    if (db < WIDE) {
      mk[db] = bk;
      mc[db] = bc;
    }
    if (valid && dc < WIDE) {
      mk[dc] = key;
      mc[dc] = code;
    }
    __syncwarp(g.mask);
    bk = mk[g.c];
    bc = mc[g.c];
    __syncwarp(g.mask);
    cnt = min(cnt + __popc(m), WIDE);
    if (cnt >= WIDE) {
      kmin = gshfl(g, bk, WIDE - 1);
      ktl = fmaxf(P.t_min, key_t(kmin));
    }
  }
};

// Group sum (every lane receives the same bits).
__device__ __forceinline__ float gsum(const Grp& g, float v) {
#pragma unroll
  for (int off = WIDE / 2; off > 0; off >>= 1) v += __shfl_xor_sync(g.mask, v, off, WIDE);
  return v;
}
// Sixteen sums over the 32 lanes of a warp at once (a recursive-halving
// reduce-scatter): at offsets 8, 4, 2, 1 each lane keeps the half of its
// values whose index bit matches its own lane bit and adds its partner's
// copy of that half, then one butterfly at offset 16 completes the sums, so
// lanes k and k + 16 end with the sum of v[k]: 16 shuffles, 16 adds and 30
// selects for sixteen sums instead of 80 shuffles and 80 adds.  Lanes k and
// k + 16 add the same two partial sums, so they hold the same bits.
__device__ __forceinline__ float gsum_transposed(const Grp& g, float (&v)[16]) {
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) {
    const bool up = (g.c & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = up ? v[i] : v[i + o];
      const float keep = up ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(g.mask, send, o, WIDE);
    }
  }
  return v[0] + __shfl_xor_sync(g.mask, v[0], 16, WIDE);
}

// Multi-round k-buffer composite of one ray (Eq. 6-7 with the early stop),
// cooperative: each round collects the K nearest hits beyond the last
// round's, then composites them front to back in parallel -- transmittance
// in front of each hit by a prefix product over the lanes, the stop at the
// first hit whose transmittance behind it falls below T_min, the weighted
// sums by one reduce-scatter over the lanes.  Every lane ends with the same
// Surface.
//
// Normal and roughness are summed, like the position, as offsets from the
// first composited hit's (n_ref, r_ref): sum w n_j = W n_ref + sum w (n_j -
// n_ref), so the FP32 sums carry small terms (exactly 0 on a flat wall)
// and their rounding no longer scales with n and r themselves.
//
// Precise (the primary record, from which shading rays start and BSDF
// samples are drawn): x, n and r are assembled from the pairs and offsets
// in double-float (W / (W + eps) too, which in FP32 can land an ulp below 1
// and move x by up to ~2e-7) and returned as FP32 values plus their
// residuals (x_lo, n_lo, r_lo).  Otherwise the residuals are 0.
template <class Ray, bool Precise = false, class Cnt>
__device__ __forceinline__ void coop_composite(const Grp& g, const Inst* insts, int n_inst, float3 o, float3 olo,
                                               float3 d,
                                               const DevParams& P, const CStack& st, int* status, Cnt& cnt,
                                               Surface& s, unsigned& composited) {
  NearKCoop kb;
  kb.P = P;
  kb.mk = st.mk;
  kb.mc = st.mc;
  kb.ma = st.ma;
  kb.insts = insts;
  kb.qc = st.qc;
  const Ray ray = make_ray<Ray>(st.ray, g.c, g.mask, o, d, olo);
  // The composited position sum w x_j / (W + eps) is kept as
  // (o + t_ref d) W / (W + eps) + d sum w (t_j - t_ref) / (W + eps) around
  // the depth t_ref + tl_ref of the first composited hit (its key keeps the
  // low part): the hit points of a ray differ by little along it, so the
  // offsets stay small and the position carries about one rounding of
  // o + t_ref d instead of one per hit (shading rays start there).
  //
  // The sums are the same for every lane; lane k % WIDE keeps sum k (slot
  // k / WIDE of its acc), so across the traversal a lane holds one or two
  // registers for them instead of fifteen or more.
  enum {
    A_W, A_DT, A_T, A_NX, A_NY, A_NZ, A_AX, A_AY, A_AZ, A_M, A_R, A_TREF, A_TLREF, A_HITS, A_SKLO, A_SKHI,
    A_NXR, A_NYR, A_NZR, A_RR, NACC  // n_ref, r_ref
  };
  constexpr int NSLOT = (NACC + WIDE - 1) / WIDE;
  float acc[NSLOT];
#pragma unroll
  for (int k = 0; k < NSLOT; ++k) acc[k] = 0.0f;
  auto add = [&](int k, float v) {
    if (g.c == k % WIDE) acc[k / WIDE] += v;
  };
  auto put = [&](int k, float v) {
    if (g.c == k % WIDE) acc[k / WIDE] = v;
  };
  auto get = [&](int k) { return gshfl(g, acc[k / WIDE], k % WIDE); };
  float T = 1.0f;
  unsigned long long last = 0ull;
  bool done = false;
  for (int round = 0; round < P.max_rounds && !done; ++round) {
    kb.reset(last, T);
    coop_traverse(g, insts, n_inst, ray, kb, st, status, cnt);
    const int n = kb.cnt;
    if (n == 0) break;
    bool have = g.c < n;
    if (have) have = LF_IN_BOUNDS(kb.bc >> 24, n_inst, status, "hit instance") &&
                     LF_IN_BOUNDS(kb.bc & 0xffffff, insts[kb.bc >> 24].n_leaves, status, "hit surfel");
    // depth and alpha~ of each entry as the hit test computed them
    const float alpha = have ? kb.ba : 0.0f, t = have ? key_t(kb.bk) : 0.0f;
    float mtl = 0.0f, rgh = 0.0f;
    float3 nj = f3(0.f, 0.f, 0.f), alb = nj;
    if (have) {
      const Inst& I = insts[kb.bc >> 24];
      const int l = kb.bc & 0xffffff;
      const int nl = I.n_leaves;
      const float4 g0 = __ldg(I.geo + l), g1 = __ldg(I.geo + nl + l), g3 = __ldg(I.geo + 3 * nl + l);
      const float4 mt = __ldg(I.mat + l);
      const float3 nh = f3(g0.w, g1.x, g1.y);
      nj = dot3(ray.d(), nh) < 0.0f ? nh : -nh;
      alb = f3(mt.x, mt.y, mt.z);
      mtl = mt.w;
      rgh = g3.z;
    }
    // inclusive prefix product of (1 - alpha) over the lanes
    float q = have ? 1.0f - alpha : 1.0f;
#pragma unroll
    for (int off = 1; off < WIDE; off <<= 1) {
      const float v = __shfl_up_sync(g.mask, q, off, WIDE);
      if (g.c >= off) q *= v;
    }
    const float qb = __shfl_up_sync(g.mask, q, 1, WIDE);
    const float Tb = g.c == 0 ? T : T * qb;  // transmittance in front of this hit
    const float Ta = T * q;                  // behind it
    const unsigned stopm = gballot(g, have && Ta < P.T_min);
    const int lastc = stopm ? __ffs(stopm) - 1 : n - 1;
    const float w = (have && g.c <= lastc) ? Tb * alpha : 0.0f;
    // the references: the first composited hit's (read back in later
    // rounds rather than kept in registers across the walk)
    float t_ref, r_ref;
    float3 n_ref;
    if (round == 0) {
      t_ref = gshfl(g, t, 0);
      n_ref = f3(gshfl(g, nj.x, 0), gshfl(g, nj.y, 0), gshfl(g, nj.z, 0));
      r_ref = gshfl(g, rgh, 0);
      put(A_TREF, t_ref);
      put(A_TLREF, key_tl(gshfl(g, kb.bk, 0)));
      put(A_NXR, n_ref.x);
      put(A_NYR, n_ref.y);
      put(A_NZR, n_ref.z);
      put(A_RR, r_ref);
    } else {
      t_ref = get(A_TREF);
      n_ref = f3(get(A_NXR), get(A_NYR), get(A_NZR));
      r_ref = get(A_RR);
    }
    if constexpr (WIDE == 32) {
      // the eleven sums at once, ending in lane k = the sum's slot
      float v[16] = {w, w * (t - t_ref), w * t, w * (nj.x - n_ref.x), w * (nj.y - n_ref.y), w * (nj.z - n_ref.z),
                     w * alb.x, w * alb.y, w * alb.z, w * mtl, w * (rgh - r_ref), 0.f, 0.f, 0.f, 0.f, 0.f};
      static_assert(A_W == 0 && A_DT == 1 && A_T == 2 && A_NX == 3 && A_NY == 4 && A_NZ == 5 && A_AX == 6 &&
                        A_AY == 7 && A_AZ == 8 && A_M == 9 && A_R == 10,
                    "the transposed sums land in slots 0..10");
      const float sum = gsum_transposed(g, v);
      if (g.c <= A_R) acc[0] += sum;
    } else {
      add(A_W, gsum(g, w));
      add(A_NX, gsum(g, w * (nj.x - n_ref.x)));
      add(A_NY, gsum(g, w * (nj.y - n_ref.y)));
      add(A_NZ, gsum(g, w * (nj.z - n_ref.z)));
      add(A_R, gsum(g, w * (rgh - r_ref)));
      add(A_DT, gsum(g, w * (t - t_ref)));
      add(A_T, gsum(g, w * t));
      add(A_AX, gsum(g, w * alb.x));
      add(A_AY, gsum(g, w * alb.y));
      add(A_AZ, gsum(g, w * alb.z));
      add(A_M, gsum(g, w * mtl));
    }
    T = gshfl(g, Ta, lastc);
    add(A_HITS, (float)(lastc + 1));
    const unsigned long long sk = gshfl(g, kb.bk, lastc);
    put(A_SKLO, __uint_as_float((unsigned)sk));
    put(A_SKHI, __uint_as_float((unsigned)(sk >> 32)));
    done = stopm != 0u || n < WIDE;
    if (!done) {
      last = kb.kmax;
      if (round == P.max_rounds - 1 && g.c == 0) report(status, LF_ERR_ROUND_LIMIT);
    }
  }
  const int hits = (int)get(A_HITS);
  if (g.c == 0) composited += (unsigned)hits;
  const float W = get(A_W);
  const float inv = 1.0f / (W + P.eps_w);
  s.T = T;
  s.W = W;
  const float tr = get(A_TREF);
  const float3 o3 = ray.o(), olo3 = ray.olo(), d3 = ray.d();
  const float3 nr = f3(get(A_NXR), get(A_NYR), get(A_NZR));
  const float rref = get(A_RR);
  const float3 Sn = f3(get(A_NX), get(A_NY), get(A_NZ));  // sum w (n_j - n_ref)
  if constexpr (Precise) {
    // W / (W + eps) = 1 - eps / (W + eps) as a pair (the FP32 error of W only
    // moves the tiny second term)
    const float ew = P.eps_w / (W + P.eps_w);
    DF wf;
    two_sum(1.0f, -ew, wf.hi, wf.lo);
    const float lo = fmaf(get(A_DT), inv, get(A_TLREF) * wf.hi);
    // o + olo + t_ref d as h + (he + pe + olo), exact to ~1e-15 relative,
    // times W / (W + eps), plus the small offset along d
    auto axis = [&](float oc, float oloc, float dc, float& xlo) {
      float p, pe, h, he;
      two_prod(dc, tr, p, pe);
      two_sum(oc, p, h, he);
      const DF x = df_add(df_mul(wf, df_renorm(h, __fadd_rn(__fadd_rn(he, pe), oloc))), DF{__fmul_rn(dc, lo), 0.0f});
      xlo = x.lo;
      return x.hi;
    };
    s.x = f3(axis(o3.x, olo3.x, d3.x, s.x_lo.x), axis(o3.y, olo3.y, d3.y, s.x_lo.y),
             axis(o3.z, olo3.z, d3.z, s.x_lo.z));
    // r = r_ref W / (W + eps) + sum w (r_j - r_ref) / (W + eps)
    const DF rr = df_add(df_mul(DF{rref, 0.0f}, wf), DF{get(A_R) * inv, 0.0f});
    s.r = rr.hi;
    s.r_lo = rr.lo;
    // n = v / |v| with v = n_ref + sum w (n_j - n_ref) / W
    if (W > 0.0f) {
      const float iw = 1.0f / W;
      DF vx, vy, vz;
      two_sum(nr.x, Sn.x * iw, vx.hi, vx.lo);
      two_sum(nr.y, Sn.y * iw, vy.hi, vy.lo);
      two_sum(nr.z, Sn.z * iw, vz.hi, vz.lo);
      const DF v2 = df_add(df_add(df_mul(vx, vx), df_mul(vy, vy)), df_mul(vz, vz));
      const DF vl = df_sqrt(v2);
      s.nlen = vl.hi * wf.hi;
      const DF nx = df_div(vx, vl), ny = df_div(vy, vl), nz = df_div(vz, vl);
      s.n = f3(nx.hi, ny.hi, nz.hi);
      s.n_lo = f3(nx.lo, ny.lo, nz.lo);
    } else {
      s.nlen = 0.0f;
    }
    if (!(s.nlen >= 1e-12f)) {
      s.n = -d3;
      s.n_lo = f3(0.f, 0.f, 0.f);
    }
  } else {
    // o + t_ref d as an exact pair (TwoProd, TwoSum), so the position is
    // rounded once, at the end
    const float wf = W * inv, lo = fmaf(get(A_DT), inv, get(A_TLREF) * wf);
    auto axis = [&](float oc, float oloc, float dc) {
      float p, pe, h, he;
      two_prod(dc, tr, p, pe);
      two_sum(oc, p, h, he);
      return fmaf(wf, h, fmaf(wf, he + pe + oloc, dc * lo));
    };
    s.x = f3(axis(o3.x, olo3.x, d3.x), axis(o3.y, olo3.y, d3.y), axis(o3.z, olo3.z, d3.z));
    s.x_lo = f3(0.f, 0.f, 0.f);
    s.r = fmaf(rref, wf, get(A_R) * inv);
    s.r_lo = 0.0f;
    const float3 mv = nr * wf + Sn * inv;
    s.nlen = sqrtf(dot3(mv, mv));
    s.n = s.nlen < 1e-12f ? -d3 : mv * (1.0f / s.nlen);
    s.n_lo = f3(0.f, 0.f, 0.f);
  }
  const float3 Sa = f3(get(A_AX), get(A_AY), get(A_AZ));
  s.depth = get(A_T) * inv;
  s.a = Sa * inv;
  s.Sa = Sa;
  s.m = get(A_M) * inv;
  s.hits = hits;
  s.stop_key = ((unsigned long long)__float_as_uint(get(A_SKHI)) << 32) | __float_as_uint(get(A_SKLO));
}

}  // namespace lf
