// Context object behind the opaque sr_ctx handle.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <array>
#include <map>
#include <string>

#include "../../include/semiring.h"

namespace sr {
constexpr int kDefaultSpinLimit = 1 << 22;
struct ServeState;
}  // namespace sr

struct sr_ctx {
    int device = 0;
    void *ws = nullptr;           // device workspace (sr_config.workspace_bytes)
    size_t ws_bytes = 0;
    int *d_status = nullptr;      // device status words: [0] error code, [1] where
    int spin_limit = sr::kDefaultSpinLimit;
    int bool_tc_mode = 1;         // tensor-core Boolean products: 0 never, 1 when K >= 1024, 2 when possible
    int bool_m4r_mode = 1;        // Four Russians Boolean products: 0 never, 1 large products, 2 always
    int closure_width = 0;        // anti-distance closure block width: 0 automatic, 128, 256, 512
    int closure_persistent = 1;   // persistent closure: 0 never, 1 large D, 2 whenever possible
    int closure_share = 128;      // persistent closure: phase-3 share before the next panels (/256)
    int bool_side_sms = -1;       // Boolean tensor-core closure: SMs phase 3 leaves to the diagonal chain (-1: default)
    int closure_fused = 1;        // fused-pass closure: 0 never, 1 automatic, 2 whenever possible
    int product_split = 1;        // deep u8/u16 products: last wave split along K in clusters (0 never, 1 auto)
    sr::ServeState *serve = nullptr;
    std::map<std::string, std::array<int, 3>> tune;   // autotuned batch configurations by signature
    // autotuned single-call choices by "op/dtype/D bucket": [choice, 0, 0, ms] (tune.cu)
    std::map<std::string, std::array<double, 4>> tuned;
    std::string tune_path;                            // JSON cache (sr_config.tune_cache), "" for none
};

namespace sr {
void sr_ctx_shutdown(sr_ctx *c);   // stops the serving loop if running
}
