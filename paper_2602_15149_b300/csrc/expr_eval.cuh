// User-defined expressions (Sec. 3.3): the bytecode and its device interpreter.
//
// The host compiler (expr_compile.h) turns an expression and its locals into a program for a small
// stack machine: postfix arithmetic on doubles, with a skip flag carried by every stack value and
// forward jumps for the lazily evaluated if(c, a, b).  An operation on a skipped operand gives a
// skipped result, an if() with a skipped condition is skipped, and only the branch it takes runs.
// Programs are checked on the host (stack depth, local and constant indices, jumps strictly forward)
// before they are uploaded, so the interpreter's loop ends after at most ncode instructions.
#pragma once
#include <stdint.h>

namespace tl {

struct ExInstr {
    uint8_t op;  // ExOp
    uint8_t a;   // variable, local or function index
    uint16_t b;  // constant index or jump target (instruction index within the program)
};

enum ExOp : uint8_t {
    EX_END = 0,
    EX_CONST,  // push consts[b]
    EX_VAR,    // push vars[a]
    EX_LOAD,   // push locals[a]
    EX_STORE,  // locals[a] = pop
    EX_SKIP,   // push a skipped value
    EX_NEG,
    EX_FN,     // top = f_a(top)
    EX_JZ,     // pop c: skipped -> push a skipped value and go to the if's end (the jump before b);
               //        c == 0 -> go to b (the else branch)
    EX_JMP,    // go to b
    // binary operators: pop b, pop a, push a op b
    EX_ADD, EX_SUB, EX_MUL, EX_DIV, EX_POW,
    EX_LT, EX_GT, EX_LE, EX_GE, EX_EQ, EX_NE, EX_AND, EX_OR,
    EX_NUM_OPS
};

// functions of the expression language, indices of EX_FN
enum ExFn : uint8_t { EXF_SIN, EXF_COS, EXF_TAN, EXF_COT, EXF_SINH, EXF_COSH, EXF_TANH, EXF_COTH, EXF_SQRT, EXF_ABS,
                      EXF_LOG, EXF_LN, EXF_NUM };

// built-in variables, in this order: x0 y0 z0 x y z ux uy uz t dt dx
constexpr int kExVars = 12;
constexpr int kExMaxStack = 24;
constexpr int kExMaxLocals = 24;

// A program within the uploaded tables: code offset, instruction count, constant offset.
struct ExProg {
    int code, ncode, consts, pad;
};

__device__ __forceinline__ double ex_fn(int f, double x) {
    switch (f) {
    case EXF_SIN: return sin(x);
    case EXF_COS: return cos(x);
    case EXF_TAN: return tan(x);
    case EXF_COT: return 1.0 / tan(x);
    case EXF_SINH: return sinh(x);
    case EXF_COSH: return cosh(x);
    case EXF_TANH: return tanh(x);
    case EXF_COTH: return 1.0 / tanh(x);
    case EXF_SQRT: return sqrt(x);
    case EXF_ABS: return fabs(x);
    case EXF_LOG: return log10(x);
    default: return log(x);
    }
}

__device__ __forceinline__ double ex_binary(int op, double a, double b) {
    switch (op) {
    case EX_ADD: return a + b;
    case EX_SUB: return a - b;
    case EX_MUL: return a * b;
    case EX_DIV: return a / b;
    case EX_POW: return pow(a, b);
    case EX_LT: return a < b ? 1.0 : 0.0;
    case EX_GT: return a > b ? 1.0 : 0.0;
    case EX_LE: return a <= b ? 1.0 : 0.0;
    case EX_GE: return a >= b ? 1.0 : 0.0;
    case EX_EQ: return a == b ? 1.0 : 0.0;
    case EX_NE: return a != b ? 1.0 : 0.0;
    case EX_AND: return (a != 0.0 && b != 0.0) ? 1.0 : 0.0;
    default: return (a != 0.0 || b != 0.0) ? 1.0 : 0.0;
    }
}

// Runs one program on one set of variables; returns its value and sets skip.
__device__ inline double ex_run(const ExInstr *code, int ncode, const double *K, const double *vars, bool &skip) {
    double st[kExMaxStack], loc[kExMaxLocals];
    uint32_t sk = 0, lsk = 0;  // skip bits of the stack slots and of the locals
    int sp = 0, pc = 0;
    while (pc < ncode) {
        const ExInstr I = code[pc++];
        switch (I.op) {
        case EX_CONST:
            st[sp] = K[I.b];
            sk &= ~(1u << sp);
            sp++;
            break;
        case EX_VAR:
            st[sp] = vars[I.a];
            sk &= ~(1u << sp);
            sp++;
            break;
        case EX_LOAD:
            st[sp] = loc[I.a];
            sk = (sk & ~(1u << sp)) | (((lsk >> I.a) & 1u) << sp);
            sp++;
            break;
        case EX_STORE:
            sp--;
            loc[I.a] = st[sp];
            lsk = (lsk & ~(1u << I.a)) | (((sk >> sp) & 1u) << I.a);
            break;
        case EX_SKIP:
            st[sp] = 0.0;
            sk |= 1u << sp;
            sp++;
            break;
        case EX_NEG: st[sp - 1] = -st[sp - 1]; break;
        case EX_FN: st[sp - 1] = ex_fn(I.a, st[sp - 1]); break;
        case EX_JZ:
            sp--;
            if ((sk >> sp) & 1u) {  // skipped condition: the whole if() is skipped
                st[sp] = 0.0;
                sk |= 1u << sp;
                sp++;
                pc = code[I.b - 1].b;
            } else if (st[sp] == 0.0) {
                pc = I.b;
            }
            break;
        case EX_JMP: pc = I.b; break;
        case EX_END: pc = ncode; break;
        default: {
            sp--;
            const uint32_t sb = (sk >> sp) & 1u;
            st[sp - 1] = ex_binary(I.op, st[sp - 1], st[sp]);
            sk |= sb << (sp - 1);
        }
        }
    }
    skip = (sk >> (sp - 1)) & 1u;
    return st[sp - 1];
}

// Evaluates program `prog` for n rows of variables (row-major, kExVars per row).
__global__ void k_expr_rows(const ExInstr *code, const double *K, ExProg prog, int64_t n, const double *vars,
                            double *out, uint8_t *skip) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double v[kExVars];
    for (int q = 0; q < kExVars; q++) v[q] = vars[r * kExVars + q];
    bool s;
    out[r] = ex_run(code + prog.code, prog.ncode, K + prog.consts, v, s);
    skip[r] = s ? 1 : 0;
}

}  // namespace tl
