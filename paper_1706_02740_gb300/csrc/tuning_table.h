// The table of tuned launch geometries (sft_tuning_table_* in sft.h), for the batch code.
#pragma once

#include <stdint.h>

#include "../../include/sft.h"

namespace sft {

// A batch's shape class: floor(log2 N), floor(log2 s), kappa and precision.
struct TuneKey {
  int32_t log2n, log2s, kappa, prec;
};

TuneKey tune_key(int64_t N, int32_t s, int32_t kappa, int32_t prec);
bool same_key(const TuneKey& a, const TuneKey& b);
bool tuning_table_find(const TuneKey& k, sft_tuning* out);
void tuning_table_store(const TuneKey& k, const sft_tuning& t);

}  // namespace sft
