// sections.cpp -- box and box-set algebra for array sections (Sec. 2.1, Sec. 4.2).
#include "sections.h"

#include <algorithm>

namespace hda {

Box make_box(int64_t lo0, int64_t lo1, int64_t lo2, int64_t hi0, int64_t hi1, int64_t hi2)
{
    Box b;
    b.lo[0] = lo0;
    b.lo[1] = lo1;
    b.lo[2] = lo2;
    b.hi[0] = hi0;
    b.hi[1] = hi1;
    b.hi[2] = hi2;
    return b;
}

Box box_intersect(const Box &a, const Box &b)
{
    Box r;
    for (int d = 0; d < 3; d++) {
        r.lo[d] = std::max(a.lo[d], b.lo[d]);
        r.hi[d] = std::min(a.hi[d], b.hi[d]);
    }
    return r;
}

bool box_overlaps(const Box &a, const Box &b)
{
    for (int d = 0; d < 3; d++)
        if (std::max(a.lo[d], b.lo[d]) >= std::min(a.hi[d], b.hi[d])) return false;
    return true;
}

bool box_contains(const Box &outer, const Box &inner)
{
    if (inner.empty()) return true;
    for (int d = 0; d < 3; d++)
        if (inner.lo[d] < outer.lo[d] || inner.hi[d] > outer.hi[d]) return false;
    return true;
}

Box box_hull(const Box &a, const Box &b)
{
    if (a.empty()) return b;
    if (b.empty()) return a;
    Box r;
    for (int d = 0; d < 3; d++) {
        r.lo[d] = std::min(a.lo[d], b.lo[d]);
        r.hi[d] = std::max(a.hi[d], b.hi[d]);
    }
    return r;
}

int64_t set_volume(const BoxSet &s)
{
    int64_t v = 0;
    for (const Box &b : s) v += b.volume();
    return v;
}

Box set_bbox(const BoxSet &s)
{
    Box r = make_box(0, 0, 0, 0, 0, 0);
    for (const Box &b : s) r = box_hull(r, b);
    return r;
}

// a - b for two boxes: at most six disjoint pieces.
static void box_subtract(const Box &a, const Box &b, BoxSet &out)
{
    if (!box_overlaps(a, b)) {
        out.push_back(a);
        return;
    }
    Box rest = a;
    for (int d = 0; d < 3; d++) {
        if (rest.lo[d] < b.lo[d]) {
            Box piece = rest;
            piece.hi[d] = b.lo[d];
            out.push_back(piece);
            rest.lo[d] = b.lo[d];
        }
        if (rest.hi[d] > b.hi[d]) {
            Box piece = rest;
            piece.lo[d] = b.hi[d];
            out.push_back(piece);
            rest.hi[d] = b.hi[d];
        }
    }
    // what remains of `rest` lies inside b and is dropped
}

void set_normalize(BoxSet &s)
{
    s.erase(std::remove_if(s.begin(), s.end(), [](const Box &b) { return b.empty(); }), s.end());
    bool merged = true;
    while (merged && s.size() > 1) {
        merged = false;
        for (int d = 2; d >= 0; d--) {
            const int e = (d + 1) % 3, f = (d + 2) % 3;
            std::sort(s.begin(), s.end(), [&](const Box &x, const Box &y) {
                if (x.lo[e] != y.lo[e]) return x.lo[e] < y.lo[e];
                if (x.hi[e] != y.hi[e]) return x.hi[e] < y.hi[e];
                if (x.lo[f] != y.lo[f]) return x.lo[f] < y.lo[f];
                if (x.hi[f] != y.hi[f]) return x.hi[f] < y.hi[f];
                return x.lo[d] < y.lo[d];
            });
            BoxSet out;
            out.reserve(s.size());
            for (const Box &b : s) {
                if (!out.empty()) {
                    Box &p = out.back();
                    if (p.lo[e] == b.lo[e] && p.hi[e] == b.hi[e] && p.lo[f] == b.lo[f] &&
                        p.hi[f] == b.hi[f] && p.hi[d] == b.lo[d]) {
                        p.hi[d] = b.hi[d];
                        merged = true;
                        continue;
                    }
                }
                out.push_back(b);
            }
            s.swap(out);
        }
    }
    std::sort(s.begin(), s.end());
}

BoxSet set_intersect_box(const BoxSet &a, const Box &b)
{
    BoxSet r;
    if (b.empty()) return r;
    for (const Box &x : a) {
        Box y = box_intersect(x, b);
        if (!y.empty()) r.push_back(y);
    }
    set_normalize(r);
    return r;
}

BoxSet set_intersect(const BoxSet &a, const BoxSet &b)
{
    BoxSet r;
    if (a.empty() || b.empty()) return r;
    Box ba = set_bbox(a), bb = set_bbox(b);
    if (!box_overlaps(ba, bb)) return r;
    for (const Box &x : a) {
        if (!box_overlaps(x, bb)) continue;
        for (const Box &y : b) {
            Box z = box_intersect(x, y);
            if (!z.empty()) r.push_back(z);
        }
    }
    set_normalize(r);
    return r;
}

BoxSet set_subtract(const BoxSet &a, const BoxSet &b)
{
    if (a.empty() || b.empty()) return a;
    Box bb = set_bbox(b);
    BoxSet cur;
    for (const Box &x : a) {
        if (!box_overlaps(x, bb)) {
            cur.push_back(x);
            continue;
        }
        BoxSet pieces{x};
        for (const Box &y : b) {
            if (pieces.empty()) break;
            BoxSet next;
            for (const Box &p : pieces) box_subtract(p, y, next);
            pieces.swap(next);
        }
        cur.insert(cur.end(), pieces.begin(), pieces.end());
    }
    set_normalize(cur);
    return cur;
}

BoxSet set_union(const BoxSet &a, const BoxSet &b)
{
    BoxSet r = a;
    BoxSet extra = set_subtract(b, a);
    r.insert(r.end(), extra.begin(), extra.end());
    set_normalize(r);
    return r;
}

BoxSet set_from_boxes(const std::vector<Box> &boxes)
{
    BoxSet r;
    for (const Box &b : boxes) {
        if (b.empty()) continue;
        BoxSet add = set_subtract(BoxSet{b}, r);
        r.insert(r.end(), add.begin(), add.end());
    }
    set_normalize(r);
    return r;
}

bool set_equal(const BoxSet &a, const BoxSet &b)
{
    if (a.size() == b.size()) {
        bool same = true;
        for (size_t i = 0; i < a.size() && same; i++) same = a[i] == b[i];
        if (same) return true;
    }
    if (set_volume(a) != set_volume(b)) return false;
    return set_subtract(a, b).empty();
}

bool set_overlaps(const BoxSet &a, const BoxSet &b)
{
    for (const Box &x : a)
        for (const Box &y : b)
            if (box_overlaps(x, y)) return true;
    return false;
}

bool set_contains(const BoxSet &outer, const BoxSet &inner)
{
    return set_subtract(inner, outer).empty();
}

Box offset_box(const Box &work, const int32_t o[3], const int64_t n[3])
{
    Box r;
    if (work.empty()) return make_box(0, 0, 0, 0, 0, 0);
    for (int d = 0; d < 3; d++) {
        if (o[d] == OFFSET_ALL) {
            r.lo[d] = 0;
            r.hi[d] = n[d];
        } else {
            r.lo[d] = std::max<int64_t>(work.lo[d] + o[d], 0);
            r.hi[d] = std::min<int64_t>(work.hi[d] + o[d], n[d]);
        }
    }
    return r;
}

static int64_t floor_div(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

bool trapezoid_boxes(const int64_t c[8], BoxSet *out)
{
    const int64_t top = c[0], bottom = c[4];
    if (c[0] != c[2] || c[4] != c[6] || top > bottom) return false;
    BoxSet s;
    for (int64_t r = top; r <= bottom; r++) {
        int64_t L, R;
        if (bottom == top) {
            L = c[1];
            R = c[3];
        } else {
            L = c[1] + floor_div((r - top) * (c[5] - c[1]), bottom - top);
            R = c[3] + floor_div((r - top) * (c[7] - c[3]), bottom - top);
        }
        if (L <= R) s.push_back(make_box(r, L, 0, r + 1, R + 1, 1));
    }
    set_normalize(s);
    *out = s;
    return true;
}

}  // namespace hda
