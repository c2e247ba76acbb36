// Cooperative traversal of the wide BVH: WIDE consecutive lanes of a warp
// trace one ray together (sm_103a).
//
// At a wide node lane c tests child slot c (one 32-byte slot per lane, so a
// node is one coalesced 16 * 32 B read), the group continues with the nearest
// child it enters and pushes the others on the ray's stack in shared memory;
// at a leaf lane c tests surfel first + c.  Every branch below is uniform over
// the group, so the lanes of a ray never diverge from one another and a warp
// holds 32 / WIDE rays.  Stack entries carry the entry distance of their box:
// an entry beyond the visitor's current far bound is dropped when popped.
#pragma once
#include "lf_common.cuh"

namespace lf {

constexpr int CSTACK = 128;  // stack entries per ray (each node visit pushes at most WIDE - 1)
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

// Per-ray stack (three parallel arrays in shared memory).
struct CStack {
  int* code;
  int* cnt;
  float* t;
};

// Stack entries name (instance, wide node or leaf) as in the binary
// traversal: instance << 25 | leaf flag (bit 24) | index; the leaf's surfel
// count sits in the parallel `cnt` array.
__device__ __forceinline__ int wentry(int ii, int code) {
  return code >= 0 ? ((ii << 25) | code) : ((ii << 25) | LEAF_BIT | ~code);
}

// Visitor interface (all members group-uniform except inside leaf()):
//   tlo(), thi()  culling interval of the ray
//   leaf(g, ii, first, count, I)  lanes c < count handle surfel first + c
//   done(), abort()
template <class V>
__device__ __forceinline__ void coop_traverse(const Grp& g, const Inst* insts, int n_inst, const Ray& ray, V& vis,
                                              const CStack& st, int* status, Counters& cnt) {
  int sp = 0;
  // instance boxes, WIDE at a time; instance 0 (background) ends up deepest
  for (int i0 = 0; i0 < n_inst; i0 += WIDE) {
    const int ii = i0 + g.c;
    bool hit = false;
    float tn = 0.0f;
    int code = 0, count = 0;
    if (ii < n_inst) {
      const Inst& I = insts[ii];
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
  }
  __syncwarp(g.mask);
  // a tree of n leaves has fewer than n wide nodes; the budget only guards
  // against a malformed tree
  int budget = 8;
  for (int ii = 0; ii < n_inst; ++ii) budget += insts[ii].n_leaves;
  while (sp > 0) {
    --sp;
    const float t0 = st.t[sp];
    if (t0 > vis.thi()) continue;
    int e = st.code[sp], ec = st.cnt[sp];
    while (true) {
      const int ii = e >> 25;
      const Inst& I = insts[ii];
      if (e & LEAF_BIT) {
        if (g.c == 0) cnt.tests += ec;
        vis.leaf(g, ii, e & 0xffffff, ec, I);
        if (vis.done()) return;
        break;
      }
      if (--budget < 0) {
        if (g.c == 0) report(status, LF_ERR_STACK);
        vis.abort();
        return;
      }
      if (g.c == 0) ++cnt.nodes;
      const float4* slot = I.wnodes + 2 * ((size_t)(e & 0xffffff) * WIDE + g.c);
      const float4 A = __ldg(slot), Bx = __ldg(slot + 1);
      const int code = __float_as_int(A.w), count = __float_as_int(Bx.w);
      float tn = 0.0f;
      const bool hit = code != INT_MIN && slab(A.x, A.y, A.z, Bx.x, Bx.y, Bx.z, ray, vis.tlo(), vis.thi(), tn);
      const unsigned m = gballot(g, hit);
      if (m == 0u) break;
      // nearest child: smallest entry distance (positive floats order as their bits)
      const unsigned key = hit ? __float_as_uint(tn) : 0xffffffffu;
      const unsigned kmin = __reduce_min_sync(g.mask, key);
      const int near = __ffs(gballot(g, hit && key == kmin)) - 1;
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
}

// Shadow ray (cooperative): V = prod(1 - alpha~) over all accepted hits; 0
// once below T_min.  The product of a leaf's factors is formed over the
// group by a butterfly, which leaves every lane with the same bits.
struct ShadowCoop {
  float V;
  bool stop;
  float3 o, d;
  DevParams P;
  __device__ __forceinline__ float tlo() const { return P.t_min; }
  __device__ __forceinline__ float thi() const { return BIG_F; }
  __device__ __forceinline__ bool done() const { return stop; }
  __device__ __forceinline__ void abort() { stop = true; }
  __device__ __forceinline__ void leaf(const Grp& g, int, int first, int count, const Inst& I) {
    float f = 1.0f;
    if (g.c < count) {
      const Rec r = load_rec(I.geo, first + g.c);
      float t, tl, alpha;
      if (hit_surfel(r, o, d, P, t, tl, alpha)) f = 1.0f - alpha;
    }
#pragma unroll
    for (int off = WIDE / 2; off > 0; off >>= 1) f *= __shfl_xor_sync(g.mask, f, off, WIDE);
    V *= f;
    if (V < P.T_min) {
      V = 0.0f;
      stop = true;
    }
  }
};

}  // namespace lf
