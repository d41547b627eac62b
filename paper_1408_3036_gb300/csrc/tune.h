// Launch-shape autotuner (tune.cu): candidates of a launch parameter that
// changes speed only, timed on first use per problem shape, the choice kept
// for the process and in a JSON cache file.
#pragma once

#include <string>
#include <vector>

namespace gw {

// The candidate to launch for this shape: the cached or decided one, else the
// least-sampled candidate (or cand[0] when tuning is off).
int tune_pick(const std::string& key, const std::vector<int>& cand, bool enabled);
// One timed sample (cost: milliseconds per unit of work) of the candidate.
void tune_report(const std::string& key, int choice, double cost);
// The decided candidate for this shape, or 0.
int tune_known(const std::string& key);

}  // namespace gw
