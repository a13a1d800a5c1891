// Host-only structural check of a tile plan (plan_check.cpp).
#pragma once
#include <string>

#include "tile.cuh"

namespace wdb {

// Empty string when plan P of layout L keeps its invariants: every output of every subband
// produced by exactly one item (the parts of a split tile chain its batches once), every
// staged region and tap area inside the staging buffer, every staged read of a tap inside
// its pair's region (its polyphase plane for down pairs), and the conditions of super tiles,
// split tiles and 16-byte staging; else the first fault found.
std::string check_tile_plan(const Layout& L, const TilePlanHost& P);

}  // namespace wdb
