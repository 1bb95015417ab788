// Capacities and status codes of the per-cell Voronoi construction (the
// warp-cooperative builder in voronoi_warp.cuh): planes and vertices a cell
// may hold, the cap on the staged nearest-neighbour count, and the bits a
// failing cell reports.
#pragma once

namespace emv {

constexpr int MAXP = 64;         // planes per cell (6 walls + cutting bisectors)
constexpr int MAXV = 128;        // vertices per cell
constexpr int MAXV_FIRST = 64;   // vertices per cell in the first pass (cells that need more are rebuilt)
constexpr int MAXK = 64;         // cap on em_params.knn_k

enum : int {
    VS_OK = 0, VS_CAPACITY = 1, VS_TOPOLOGY = 2, VS_COINCIDENT = 4, VS_OUTSIDE = 8, VS_BOUNDS = 16,
    VS_CANDIDATES = 64, VS_ROUNDS = 128
};

}  // namespace emv
