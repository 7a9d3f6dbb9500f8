// local.cuh -- the canonical zd-tree in pointer form, updated point by point
// (Sec. 2 "Batch-dynamic updates", Algorithm 4, and the deletion the paper
// says uses an almost identical algorithm), for batches too small to pay for
// re-deriving the whole flat tree.
//
// Internal nodes and leaves live in pools; every leaf keeps its points in a
// slab of (key, point) entries sorted by (key, id).  Inserting a point walks
// down by key bits (Algorithm 4's descent), makes a new internal node where
// the key leaves a node's prefix (the cut that was pruned there, Sec. 2.1, is
// no longer empty) and splits a leaf that grows past L on the highest bit
// where its keys differ (Algorithm 1's split).  Deleting a point splices out
// a leaf that becomes empty and collapses the topmost subtree whose size
// drops to L into one leaf.  After every point the structure is exactly the
// canonical tree of the current point set: a node is a leaf iff it holds at
// most L points or all its keys are equal, and an internal node splits on the
// highest differing bit of its keys.  Sizes and tight boxes are kept on the
// path.  Work per point is O(depth + L) (+ the slab of a leaf of equal keys).
//
// The functions are sequential: one device thread applies one small batch.
// The same code compiles for the host, so the tests check it against the
// oracle without a GPU.  Pools and slab storage are bump-allocated; what a
// collapse or splice frees is not reused until the pointer form is rebuilt
// from the flat tree.  Every operation checks first that the pools hold what
// it may need and reports LT_NO_SPACE, leaving the tree unchanged, otherwise.
#pragma once

#include <stdint.h>

#ifndef __CUDACC__
#ifndef __host__
#define __host__
#endif
#ifndef __device__
#define __device__
#endif
#ifndef __forceinline__
#define __forceinline__ inline
#endif
#endif

namespace zdlocal {

typedef unsigned long long u64;

struct P4 {
    int x, y, z, w; // coordinates and id (same layout as the flat tree's int4)
};

// Reference to a node: >= 0 internal node i, < 0 leaf ~j, LT_EMPTY none.
constexpr int LT_EMPTY = -2147483647 - 1;
constexpr int LT_MAX_DEPTH = 72; // > key bits + 1

struct LNode {
    u64 key; // a key of the node: all its keys share the bits above `bit`
    int left, right, parent;
    int bit;  // split bit
    int size; // points below
    int pad;
    P4 lo, hi; // tight box (w unused)
};

struct LLeaf {
    int parent;
    int size; // -1: a leaf that a splice or collapse removed from the tree
    int cap; // slab capacity
    int pad;
    int64_t off; // slab start in the entry storage
    P4 lo, hi;
};

struct LLoc {
    int leaf, slot;
};

// Device-resident counters of one pointer-form tree.
struct LCounters {
    int root;
    int n_nodes, n_leaves; // pool entries handed out
    int count;             // points
    int64_t stor_used;     // slab entries handed out
    int state;             // 0: in step with the point set; 1: fell back (see local.cu)
    int log_n;             // entries of the fallback log
};

enum { LT_OK = 0, LT_NO_SPACE = 1 };

struct LocalTree {
    int L;
    LNode *nodes;
    int node_cap;
    LLeaf *leaves;
    int leaf_cap;
    u64 *skeys; // slab entries: keys
    P4 *spts;   // slab entries: points
    int64_t stor_cap;
    LLoc *loc; // per id: leaf and slot
    LCounters *ctr;
};

__host__ __device__ __forceinline__ int clz64(u64 x)
{
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

__host__ __device__ __forceinline__ int imin(int a, int b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int imax(int a, int b) { return a > b ? a : b; }

__host__ __device__ __forceinline__ P4 box_empty_lo() { return P4{2147483647, 2147483647, 2147483647, 0}; }
__host__ __device__ __forceinline__ P4 box_empty_hi() { return P4{-2147483647 - 1, -2147483647 - 1, -2147483647 - 1, 0}; }
__host__ __device__ __forceinline__ P4 pmin(P4 a, P4 b) { return P4{imin(a.x, b.x), imin(a.y, b.y), imin(a.z, b.z), 0}; }
__host__ __device__ __forceinline__ P4 pmax(P4 a, P4 b) { return P4{imax(a.x, b.x), imax(a.y, b.y), imax(a.z, b.z), 0}; }

// (key, id) order of entries
__host__ __device__ __forceinline__ bool entry_less(u64 ka, int ia, u64 kb, int ib)
{
    return ka < kb || (ka == kb && ia < ib);
}

// ------------------------------------------------------------- node access
__host__ __device__ __forceinline__ int parent_of(const LocalTree &t, int ref)
{
    return ref >= 0 ? t.nodes[ref].parent : t.leaves[~ref].parent;
}
// First sorted position of live leaf j: the leaves in key order are the
// in-order leaves, so it is the number of points in the left subtrees that
// the path from the leaf to the root passes on their right.
__host__ __device__ __forceinline__ int64_t leaf_position(const LocalTree &t, int j)
{
    int64_t pos = 0;
    int child = ~j;
    int p = t.leaves[j].parent;
    for (int d = 0; p >= 0 && d < LT_MAX_DEPTH; p = t.nodes[p].parent, ++d) {
        const LNode &nd = t.nodes[p];
        if (nd.right == child) pos += nd.left >= 0 ? t.nodes[nd.left].size : t.leaves[~nd.left].size;
        child = p;
    }
    return pos;
}

__host__ __device__ __forceinline__ void set_parent(LocalTree &t, int ref, int p)
{
    if (ref >= 0) t.nodes[ref].parent = p;
    else t.leaves[~ref].parent = p;
}
__host__ __device__ __forceinline__ P4 lo_of(const LocalTree &t, int ref)
{
    return ref >= 0 ? t.nodes[ref].lo : t.leaves[~ref].lo;
}
__host__ __device__ __forceinline__ P4 hi_of(const LocalTree &t, int ref)
{
    return ref >= 0 ? t.nodes[ref].hi : t.leaves[~ref].hi;
}
__host__ __device__ __forceinline__ int size_of(const LocalTree &t, int ref)
{
    return ref >= 0 ? t.nodes[ref].size : t.leaves[~ref].size;
}

// Put `nw` where `old` hung below p (p < 0: at the root).
__host__ __device__ __forceinline__ void replace_child(LocalTree &t, int p, int old, int nw)
{
    if (p < 0) {
        t.ctr->root = nw;
    } else if (t.nodes[p].left == old) {
        t.nodes[p].left = nw;
    } else {
        t.nodes[p].right = nw;
    }
    set_parent(t, nw, p);
}

// ------------------------------------------------------------ allocation
__host__ __device__ __forceinline__ int new_node(LocalTree &t)
{
    const int i = t.ctr->n_nodes++;
    return i;
}

// A leaf with an empty slab of `cap` entries.
__host__ __device__ __forceinline__ int new_leaf(LocalTree &t, int cap)
{
    const int j = t.ctr->n_leaves++;
    LLeaf &f = t.leaves[j];
    f.parent = -1;
    f.size = 0;
    f.cap = cap;
    f.pad = 0;
    f.off = t.ctr->stor_used;
    t.ctr->stor_used += cap;
    f.lo = box_empty_lo();
    f.hi = box_empty_hi();
    return j;
}

__host__ __device__ __forceinline__ bool have_room(const LocalTree &t, int nodes, int leaves, int64_t entries)
{
    return t.ctr->n_nodes + nodes <= t.node_cap && t.ctr->n_leaves + leaves <= t.leaf_cap &&
           t.ctr->stor_used + entries <= t.stor_cap;
}

// Capacity of a new slab holding `size` entries: room for L + 1 more (a
// leaf reaches L + 1 entries before it splits).
__host__ __device__ __forceinline__ int slab_cap(const LocalTree &t, int size) { return size + t.L + 1; }

// ------------------------------------------------------------------ slabs
__host__ __device__ __forceinline__ void leaf_box(LocalTree &t, int j)
{
    LLeaf &f = t.leaves[j];
    P4 lo = box_empty_lo(), hi = box_empty_hi();
    for (int r = 0; r < f.size; ++r) {
        lo = pmin(lo, t.spts[f.off + r]);
        hi = pmax(hi, t.spts[f.off + r]);
    }
    f.lo = lo;
    f.hi = hi;
}

// Insert an entry at its (key, id) place in leaf j's slab (room checked).
__host__ __device__ __forceinline__ void slab_insert(LocalTree &t, int j, u64 key, P4 p)
{
    LLeaf &f = t.leaves[j];
    int r = f.size;
    while (r > 0 && entry_less(key, p.w, t.skeys[f.off + r - 1], t.spts[f.off + r - 1].w)) {
        t.skeys[f.off + r] = t.skeys[f.off + r - 1];
        t.spts[f.off + r] = t.spts[f.off + r - 1];
        t.loc[t.spts[f.off + r].w] = LLoc{j, r};
        --r;
    }
    t.skeys[f.off + r] = key;
    t.spts[f.off + r] = p;
    t.loc[p.w] = LLoc{j, r};
    ++f.size;
}

__host__ __device__ __forceinline__ void slab_remove(LocalTree &t, int j, int slot)
{
    LLeaf &f = t.leaves[j];
    for (int r = slot; r + 1 < f.size; ++r) {
        t.skeys[f.off + r] = t.skeys[f.off + r + 1];
        t.spts[f.off + r] = t.spts[f.off + r + 1];
        t.loc[t.spts[f.off + r].w] = LLoc{j, r};
    }
    --f.size;
}

// Move leaf j's slab to a fresh one of capacity `cap` (slots unchanged).
__host__ __device__ __forceinline__ void slab_grow(LocalTree &t, int j, int cap)
{
    LLeaf &f = t.leaves[j];
    const int64_t off = t.ctr->stor_used;
    t.ctr->stor_used += cap;
    for (int r = 0; r < f.size; ++r) {
        t.skeys[off + r] = t.skeys[f.off + r];
        t.spts[off + r] = t.spts[f.off + r];
    }
    f.off = off;
    f.cap = cap;
}

// ------------------------------------------------------------------ insert
// Insert point p (id in p.w) with Morton key `key`.
__host__ __device__ inline int insert_point(LocalTree &t, u64 key, P4 p)
{
    LCounters &c = *t.ctr;
    const int L = t.L;
    if (c.root == LT_EMPTY) {
        if (!have_room(t, 0, 1, slab_cap(t, 1))) return LT_NO_SPACE;
        const int j = new_leaf(t, slab_cap(t, 1));
        slab_insert(t, j, key, p);
        t.leaves[j].lo = t.leaves[j].hi = P4{p.x, p.y, p.z, 0};
        c.root = ~j;
        ++c.count;
        return LT_OK;
    }
    // 1. find where the key goes, without changing anything
    int path[LT_MAX_DEPTH];
    int depth = 0;
    int v = c.root;
    bool diverge = false;
    while (v >= 0) {
        const LNode &nd = t.nodes[v];
        if (((key ^ nd.key) >> nd.bit) >> 1) { // a key bit above the split bit differs
            diverge = true;
            break;
        }
        path[depth++] = v;
        v = ((key >> nd.bit) & 1) ? nd.right : nd.left;
    }
    // 2. room for the worst case of this point
    if (diverge) {
        if (!have_room(t, 1, 1, slab_cap(t, 1))) return LT_NO_SPACE;
    } else {
        const LLeaf &f = t.leaves[~v];
        const int64_t grow = f.size + 1 > f.cap ? 2 * (int64_t)f.cap : 0;
        if (!have_room(t, 1, 1, grow + slab_cap(t, L + 1))) return LT_NO_SPACE;
    }
    // 3. apply: the visited nodes gain the point
    const P4 q{p.x, p.y, p.z, 0};
    for (int i = 0; i < depth; ++i) {
        LNode &nd = t.nodes[path[i]];
        ++nd.size;
        nd.lo = pmin(nd.lo, q);
        nd.hi = pmax(nd.hi, q);
    }
    const int parent = depth ? path[depth - 1] : -1;
    if (diverge) {
        // new internal node w above v, on the highest bit where the key
        // leaves v's prefix; the point gets a leaf of its own
        const LNode &nv = t.nodes[v];
        const int bw = 63 - clz64(key ^ nv.key);
        const int cl = new_leaf(t, slab_cap(t, 1));
        slab_insert(t, cl, key, p);
        t.leaves[cl].lo = t.leaves[cl].hi = q;
        const int w = new_node(t);
        LNode &nw = t.nodes[w];
        nw.key = nv.key;
        nw.bit = bw;
        nw.size = nv.size + 1;
        nw.pad = 0;
        nw.lo = pmin(nv.lo, q);
        nw.hi = pmax(nv.hi, q);
        if ((key >> bw) & 1) {
            nw.left = v;
            nw.right = ~cl;
        } else {
            nw.left = ~cl;
            nw.right = v;
        }
        replace_child(t, parent, v, w);
        set_parent(t, v, w);
        t.leaves[cl].parent = w;
        ++c.count;
        return LT_OK;
    }
    const int j = ~v;
    if (t.leaves[j].size + 1 > t.leaves[j].cap) slab_grow(t, j, 2 * t.leaves[j].cap);
    slab_insert(t, j, key, p);
    LLeaf &f = t.leaves[j];
    f.lo = pmin(f.lo, q);
    f.hi = pmax(f.hi, q);
    ++c.count;
    const u64 first = t.skeys[f.off], last = t.skeys[f.off + f.size - 1];
    if (f.size <= L || first == last) return LT_OK;
    // split the leaf on the highest bit where its keys differ: the first
    // entries (bit clear) stay, the rest move to a new leaf
    const int hd = 63 - clz64(first ^ last);
    int s = 0;
    while (!((t.skeys[f.off + s] >> hd) & 1)) ++s;
    const int nb = f.size - s;
    const int jb = new_leaf(t, slab_cap(t, nb));
    LLeaf &fa = t.leaves[j];
    LLeaf &fb = t.leaves[jb];
    for (int r = 0; r < nb; ++r) {
        t.skeys[fb.off + r] = t.skeys[fa.off + s + r];
        t.spts[fb.off + r] = t.spts[fa.off + s + r];
        t.loc[t.spts[fb.off + r].w] = LLoc{jb, r};
    }
    fb.size = nb;
    fa.size = s;
    leaf_box(t, j);
    leaf_box(t, jb);
    const int u = new_node(t);
    LNode &nu = t.nodes[u];
    nu.key = first;
    nu.bit = hd;
    nu.size = s + nb;
    nu.pad = 0;
    nu.lo = pmin(fa.lo, fb.lo);
    nu.hi = pmax(fa.hi, fb.hi);
    nu.left = ~j;
    nu.right = ~jb;
    replace_child(t, parent, ~j, u);
    fa.parent = u;
    fb.parent = u;
    return LT_OK;
}

// ------------------------------------------------------------------ delete
// Tight boxes of the internal nodes from `ref` up to the root.
__host__ __device__ __forceinline__ void boxes_up(LocalTree &t, int ref)
{
    for (int a = ref; a >= 0; a = t.nodes[a].parent) {
        LNode &nd = t.nodes[a];
        nd.lo = pmin(lo_of(t, nd.left), lo_of(t, nd.right));
        nd.hi = pmax(hi_of(t, nd.left), hi_of(t, nd.right));
    }
}

// Replace the subtree at internal node a (size <= L) by one leaf holding its
// points in (key, id) order (in-order leaves are in key order).
__host__ __device__ inline int collapse(LocalTree &t, int a)
{
    const int sz = t.nodes[a].size;
    const int j = new_leaf(t, slab_cap(t, sz));
    int stack[LT_MAX_DEPTH];
    int sp = 0;
    stack[sp++] = a;
    while (sp) {
        const int v = stack[--sp];
        if (v >= 0) {
            stack[sp++] = t.nodes[v].right; // left first out
            stack[sp++] = t.nodes[v].left;
        } else {
            LLeaf &src = t.leaves[~v];
            LLeaf &f = t.leaves[j];
            for (int r = 0; r < src.size; ++r) {
                t.skeys[f.off + f.size] = t.skeys[src.off + r];
                t.spts[f.off + f.size] = t.spts[src.off + r];
                t.loc[t.spts[f.off + f.size].w] = LLoc{j, f.size};
                ++f.size;
            }
            src.size = -1; // removed from the tree
        }
    }
    leaf_box(t, j);
    replace_child(t, t.nodes[a].parent, a, ~j);
    return j;
}

// Delete the point with this id (it must be in the tree).
__host__ __device__ inline int delete_point(LocalTree &t, int id)
{
    LCounters &c = *t.ctr;
    if (!have_room(t, 0, 1, slab_cap(t, t.L))) return LT_NO_SPACE;
    const LLoc lc = t.loc[id];
    const int j = lc.leaf;
    slab_remove(t, j, lc.slot);
    --c.count;
    // the ancestors lose the point; the topmost one left with at most L
    // points becomes a leaf (the ones with at most L are contiguous from the
    // bottom, since sizes grow upward)
    int top = -1;
    bool small = true;
    for (int a = t.leaves[j].parent; a >= 0; a = t.nodes[a].parent) {
        --t.nodes[a].size;
        if (small && t.nodes[a].size <= t.L) top = a;
        else small = false;
    }
    if (top >= 0) {
        const int nj = collapse(t, top);
        boxes_up(t, t.leaves[nj].parent);
        return LT_OK;
    }
    LLeaf &f = t.leaves[j];
    if (f.size > 0) {
        leaf_box(t, j);
        boxes_up(t, f.parent);
        return LT_OK;
    }
    // an empty leaf: its parent's other child takes the parent's place
    const int p = f.parent;
    f.size = -1; // removed from the tree
    if (p < 0) {
        c.root = LT_EMPTY;
        return LT_OK;
    }
    const int sib = t.nodes[p].left == ~j ? t.nodes[p].right : t.nodes[p].left;
    const int gp = t.nodes[p].parent;
    replace_child(t, gp, p, sib);
    if (gp >= 0) boxes_up(t, gp);
    return LT_OK;
}

} // namespace zdlocal
