// Host-side compiled netlist shared by the compiler and the C-ABI layer.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "diffpower.h"

namespace dp {

constexpr int kMaxArity = 4;
constexpr int kGenStart = 32;          // first generated logic id (Algorithm 1, GEN_START)
constexpr uint32_t kNetMask = 0xFFFFFFu;
constexpr int64_t kMaxNets = (1 << 24) - 1;

// Bytecode opcodes (Sec. III-A): post-order stack machine.
enum BcOp : uint8_t { BC_IN = 0, BC_NOT = 1, BC_AND = 2, BC_OR = 3, BC_XOR = 4, BC_C0 = 5, BC_C1 = 6 };

struct Function {
    std::vector<uint8_t> ops;
    std::vector<int8_t> args;
    std::vector<std::string> inputs;   // input order = first appearance (CollectInputOrder)
    uint16_t tt = 0;                   // truth table, bit m = f(m), bit j of m = input j
    int logic_id = -1;                 // common-gate id (< kGenStart) or -1
};

// Parses one expression into bytecode; returns false with a message on error.
bool compile_function(const std::string &expr, Function *f, std::string *err);

}  // namespace dp

struct dp_compiled {
    int64_t n_nets = 0, n_start = 0, n_cells = 0, n_edges = 0;
    int32_t n_levels = 0, n_ops = 0;
    std::vector<int32_t> lvl_ptr;
    std::vector<uint32_t> fanin;       // 4 per cell
    std::vector<int32_t> fout_ptr, fout_edge;
    std::vector<int32_t> edge_fpos;    // 4 per cell: position of edge (cell, slot) in fout_edge, -1 unused
    std::vector<int32_t> net_of_user, user_of_net, cell_of_user, user_of_cell;
    std::vector<float> base_cap, pincap;
    uint8_t op_arity[256] = {0};
    uint16_t op_tt[256] = {0};
    std::vector<uint8_t> bc_ops;
    std::vector<int8_t> bc_args;
    int32_t bc_offset[256];
    int32_t bc_length[256];
};
