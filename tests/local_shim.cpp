// Host build of the library's point-by-point updater (csrc/local.cuh), for
// the CPU tests: the same header the device kernel runs, driven one point at
// a time from an empty tree, with an in-order export of the canonical dump.
// Test infrastructure only.
#include <stdint.h>
#include <stdlib.h>

#include <vector>

#include "../paper_2111_04182_gb300/csrc/local.cuh"
#include "../paper_2111_04182_gb300/csrc/morton.cuh"

using namespace zdlocal;

struct Shim {
    int dim, B;
    std::vector<LNode> nodes;
    std::vector<LLeaf> leaves;
    std::vector<u64> skeys;
    std::vector<P4> spts;
    std::vector<LLoc> loc;
    LCounters ctr;
    LocalTree t;
};

extern "C" {

void *lt_new(int dim, int L, int B, int64_t id_cap, int node_cap, int leaf_cap, int64_t stor_cap)
{
    Shim *s = new Shim();
    s->dim = dim;
    s->B = B;
    s->nodes.resize(node_cap > 0 ? node_cap : 1);
    s->leaves.resize(leaf_cap > 0 ? leaf_cap : 1);
    s->skeys.resize(stor_cap > 0 ? stor_cap : 1);
    s->spts.resize(stor_cap > 0 ? stor_cap : 1);
    s->loc.resize(id_cap > 0 ? id_cap : 1);
    s->ctr = LCounters{LT_EMPTY, 0, 0, 0, 0, 0, 0};
    s->t = LocalTree{L, s->nodes.data(), node_cap, s->leaves.data(), leaf_cap, s->skeys.data(), s->spts.data(),
                     stor_cap, s->loc.data(), &s->ctr};
    return s;
}

void lt_free(void *h) { delete (Shim *)h; }

static u64 key_of(const Shim *s, const int32_t *c)
{
    if (s->dim == 3) return zdk::interleave<3>((u64)c[0], (u64)c[1], (u64)c[2]);
    return zdk::interleave<2>((u64)c[0], (u64)c[1], 0);
}

// Insert points [b, dim] with ids first_id..; stops at the first failure.
int lt_insert(void *h, const int32_t *pts, int64_t b, int32_t first_id)
{
    Shim *s = (Shim *)h;
    for (int64_t i = 0; i < b; ++i) {
        const int32_t *c = pts + i * s->dim;
        P4 p{c[0], c[1], s->dim == 3 ? c[2] : 0, (int)(first_id + i)};
        int r = insert_point(s->t, key_of(s, c), p);
        if (r != LT_OK) return r;
    }
    return LT_OK;
}

int lt_delete(void *h, const int32_t *ids, int64_t b)
{
    Shim *s = (Shim *)h;
    for (int64_t i = 0; i < b; ++i) {
        int r = delete_point(s->t, ids[i]);
        if (r != LT_OK) return r;
    }
    return LT_OK;
}

int lt_count(void *h) { return ((Shim *)h)->ctr.count; }

// In-order walk: every node as (lo, hi, bit) over sorted positions (bit -1
// for a leaf) with its box, and the points' ids and keys in sorted order.
// Also checks the stored sizes and parents and every leaf's computed first
// position; returns the node count, or -1 if one of them is inconsistent.
int64_t lt_export(void *h, int64_t *lo, int64_t *hi, int32_t *bit, int32_t *box_lo, int32_t *box_hi, int32_t *ids,
                  uint64_t *keys)
{
    Shim *s = (Shim *)h;
    LocalTree &t = s->t;
    if (s->ctr.root == LT_EMPTY) {
        for (int j = 0; j < s->ctr.n_leaves; ++j)
            if (t.leaves[j].size >= 0) return -1;
        return 0;
    }
    struct Frame {
        int ref, parent, state;
        int64_t lo, idx;
    };
    std::vector<Frame> st;
    st.push_back(Frame{s->ctr.root, -1, 0, 0, 0});
    int64_t pos = 0, nn = 0;
    bool ok = true;
    while (!st.empty()) {
        Frame &f = st.back();
        if (f.ref < 0) {
            const LLeaf &lf = t.leaves[~f.ref];
            if (lf.parent != f.parent) ok = false;
            if (leaf_position(t, ~f.ref) != pos) ok = false; // the re-derivation's placement
            const int64_t a = pos;
            for (int r = 0; r < lf.size; ++r) {
                ids[pos] = t.spts[lf.off + r].w;
                keys[pos] = t.skeys[lf.off + r];
                const LLoc l = t.loc[t.spts[lf.off + r].w];
                if (l.leaf != ~f.ref || l.slot != r) ok = false;
                ++pos;
            }
            lo[nn] = a;
            hi[nn] = pos;
            bit[nn] = -1;
            const P4 bl = lf.lo, bh = lf.hi;
            box_lo[3 * nn] = bl.x, box_lo[3 * nn + 1] = bl.y, box_lo[3 * nn + 2] = bl.z;
            box_hi[3 * nn] = bh.x, box_hi[3 * nn + 1] = bh.y, box_hi[3 * nn + 2] = bh.z;
            ++nn;
            st.pop_back();
            continue;
        }
        const LNode &nd = t.nodes[f.ref];
        if (f.state == 0) {
            if (nd.parent != f.parent) ok = false;
            f.lo = pos;
            f.idx = nn++;
            f.state = 1;
            const int l = nd.left, me = f.ref;
            st.push_back(Frame{l, me, 0, 0, 0});
        } else if (f.state == 1) {
            f.state = 2;
            const int r = nd.right, me = f.ref;
            st.push_back(Frame{r, me, 0, 0, 0});
        } else {
            const int64_t k = f.idx;
            lo[k] = f.lo;
            hi[k] = pos;
            bit[k] = nd.bit;
            if (nd.size != pos - f.lo) ok = false;
            box_lo[3 * k] = nd.lo.x, box_lo[3 * k + 1] = nd.lo.y, box_lo[3 * k + 2] = nd.lo.z;
            box_hi[3 * k] = nd.hi.x, box_hi[3 * k + 1] = nd.hi.y, box_hi[3 * k + 2] = nd.hi.z;
            st.pop_back();
        }
    }
    if (pos != s->ctr.count) ok = false;
    // the leaves not marked removed are exactly the reachable ones
    int64_t reach = 0, marked_live = 0;
    for (int64_t i = 0; i < nn; ++i) reach += bit[i] == -1;
    for (int j = 0; j < s->ctr.n_leaves; ++j) marked_live += t.leaves[j].size >= 0;
    if (reach != marked_live) ok = false;
    return ok ? nn : -1;
}

} // extern "C"
