// sections.h -- array sections as boxes and sets of disjoint boxes.
//
// A section [LB:UB] of an HDArray (Sec. 2.1) is a box: per dimension a half-open range
// [lo, hi).  GDEF, LDEF and LUSE are unions of sections (Sec. 2.1); here a set is a vector of
// pairwise disjoint boxes, kept merged (adjacent boxes that line up are fused, Sec. 5.2 reports
// merging adjacent or redundant sections) and sorted (Sec. 4.2 keeps GDEF sorted so that two sets
// compare in linear time).
//
// Coordinates are in the user's dimension order, padded to three dimensions at the back
// (unused dimensions: lo 0, hi 1).
#pragma once

#include <stdint.h>

#include <vector>

namespace hda {

struct Box {
    int64_t lo[3];
    int64_t hi[3];

    bool empty() const { return hi[0] <= lo[0] || hi[1] <= lo[1] || hi[2] <= lo[2]; }
    int64_t volume() const {
        return empty() ? 0 : (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
    }
    bool operator==(const Box &o) const {
        for (int d = 0; d < 3; d++)
            if (lo[d] != o.lo[d] || hi[d] != o.hi[d]) return false;
        return true;
    }
    bool operator<(const Box &o) const {
        for (int d = 0; d < 3; d++) {
            if (lo[d] != o.lo[d]) return lo[d] < o.lo[d];
        }
        for (int d = 0; d < 3; d++) {
            if (hi[d] != o.hi[d]) return hi[d] < o.hi[d];
        }
        return false;
    }
};

Box make_box(int64_t lo0, int64_t lo1, int64_t lo2, int64_t hi0, int64_t hi1, int64_t hi2);
Box box_intersect(const Box &a, const Box &b);
bool box_contains(const Box &outer, const Box &inner);
bool box_overlaps(const Box &a, const Box &b);
Box box_hull(const Box &a, const Box &b);  // bounding box (of non-empty boxes)

using BoxSet = std::vector<Box>;  // pairwise disjoint, non-empty

int64_t set_volume(const BoxSet &s);
Box set_bbox(const BoxSet &s);  // empty box {0..0} for an empty set

// a n b, a - b, a u b.  Inputs disjoint; outputs disjoint and normalised.
BoxSet set_intersect(const BoxSet &a, const BoxSet &b);
BoxSet set_intersect_box(const BoxSet &a, const Box &b);
BoxSet set_subtract(const BoxSet &a, const BoxSet &b);
BoxSet set_union(const BoxSet &a, const BoxSet &b);
// Union of boxes that may overlap each other.
BoxSet set_from_boxes(const std::vector<Box> &boxes);
bool set_equal(const BoxSet &a, const BoxSet &b);
bool set_overlaps(const BoxSet &a, const BoxSet &b);
bool set_contains(const BoxSet &outer, const BoxSet &inner);

// Merge boxes that are adjacent along one dimension and identical in the other two, then sort.
void set_normalize(BoxSet &s);

// Offset clause composed with a work box (Sec. 3, offset clauses): the elements w + o for w in
// the work box, for one offset o; a component equal to ALL spans the whole dimension.
// Clipped to the array extent n (offsets leaving the array touch nothing there).
constexpr int32_t OFFSET_ALL = INT32_MIN;
Box offset_box(const Box &work, const int32_t o[3], const int64_t n[3]);

// Trapezoid (Sec. 3.1, HDArraySetTrapezoidUse/Def): corners ul_r, ul_c, ur_r, ur_c, ll_r, ll_c,
// lr_r, lr_c name elements; row r spans the columns between the left and right edge lines,
// inclusive, each edge rounded down in exact integer arithmetic.  Returns false for corners that
// do not form a trapezoid with horizontal top and bottom edges.
bool trapezoid_boxes(const int64_t c[8], BoxSet *out);

}  // namespace hda
