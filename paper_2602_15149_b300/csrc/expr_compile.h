// User-defined expressions (Sec. 3.3): host compiler from text to the bytecode of expr_eval.cuh.
//
// Grammar, lowest precedence first (the paper's operator table): or, and, comparisons (< > <= >= == !=),
// + -, * /, unary minus, ^ (right-associative), then numbers, variables, locals, skip, function calls,
// if(c, a, b) and parentheses.  Unary minus binds looser than ^ and tighter than * and /.  Locals are
// "name = expression" separated by ';', compiled first and stored in order.  Every program is checked
// by verify() before use.
#pragma once
#include <cctype>
#include <cstdlib>
#include <stdexcept>
#include <string>
#include <vector>

#include "expr_eval.cuh"

namespace tl {

struct ExProgram {
    std::vector<ExInstr> code;
    std::vector<double> consts;
    int max_stack = 0;
};

class ExCompiler {
  public:
    // Compiles; on error returns false with a message naming the position.
    bool compile(const std::string &locals, const std::string &expr, ExProgram &out, std::string &err) {
        prog_ = ExProgram();
        names_.clear();
        depth_ = 0;
        try {
            size_t b = 0;
            while (b <= locals.size()) {
                size_t e = locals.find(';', b);
                if (e == std::string::npos) e = locals.size();
                std::string part = locals.substr(b, e - b);
                b = e + 1;
                if (part.find_first_not_of(" \t\r\n") == std::string::npos) continue;
                size_t eq = part.find('=');
                if (eq == std::string::npos) throw std::runtime_error("local without '=': " + part);
                std::string name = trim(part.substr(0, eq));
                if (!valid_local(name)) throw std::runtime_error("bad local name '" + name + "'");
                parse_all(part.substr(eq + 1), "local " + name);
                int slot = -1;
                for (size_t k = 0; k < names_.size(); k++)
                    if (names_[k] == name) slot = (int)k;
                if (slot < 0) {
                    if ((int)names_.size() >= kExMaxLocals) throw std::runtime_error("too many locals");
                    names_.push_back(name);
                    slot = (int)names_.size() - 1;
                }
                emit(EX_STORE, (uint8_t)slot, 0, -1);
            }
            parse_all(expr, "expression");
            emit(EX_END, 0, 0, 0);
        } catch (const std::exception &e) {
            err = e.what();
            return false;
        }
        out = prog_;
        return verify(out, err);
    }

    // Checks a program as the interpreter will run it: every path keeps the stack within bounds and ends
    // with one value, indices are in range, jumps go strictly forward.
    static bool verify(const ExProgram &p, std::string &err) {
        const int n = (int)p.code.size();
        if (n == 0 || n > 65535) return err = "empty or oversized program", false;
        std::vector<int> depth(n + 1, -1);  // stack depth before each instruction
        depth[0] = 0;
        for (int pc = 0; pc < n; pc++) {
            const ExInstr I = p.code[pc];
            int d = depth[pc];
            if (d < 0) continue;  // not reachable by falling through (a jump target is set below)
            auto flow = [&](int to, int dd) -> bool {
                if (to <= pc || to >= n) return false;  // every path ends at the final EX_END
                if (dd < 0 || dd > kExMaxStack) return false;
                if (depth[to] >= 0 && depth[to] != dd) return false;
                depth[to] = dd;
                return true;
            };
            bool ok = true;
            switch (I.op) {
            case EX_CONST: ok = I.b < p.consts.size() && flow(pc + 1, d + 1); break;
            case EX_VAR: ok = I.a < kExVars && flow(pc + 1, d + 1); break;
            case EX_LOAD: ok = I.a < kExMaxLocals && flow(pc + 1, d + 1); break;
            case EX_STORE: ok = I.a < kExMaxLocals && d >= 1 && flow(pc + 1, d - 1); break;
            case EX_SKIP: ok = flow(pc + 1, d + 1); break;
            case EX_NEG: ok = d >= 1 && flow(pc + 1, d); break;
            case EX_FN: ok = I.a < EXF_NUM && d >= 1 && flow(pc + 1, d); break;
            case EX_JZ:
                ok = d >= 1 && I.b >= 1 && I.b < n && p.code[I.b - 1].op == EX_JMP && p.code[I.b - 1].b > I.b &&
                     flow(pc + 1, d - 1) && flow(I.b, d - 1) && flow(p.code[I.b - 1].b, d);
                break;
            case EX_JMP: ok = flow(I.b, d); break;
            case EX_END: ok = d == 1 && pc == n - 1; break;
            default: ok = I.op < EX_NUM_OPS && d >= 2 && flow(pc + 1, d - 1);
            }
            if (!ok) return err = "invalid program at instruction " + std::to_string(pc), false;
        }
        if (p.code[n - 1].op != EX_END || depth[n - 1] != 1) return err = "program does not end with one value", false;
        return true;
    }

  private:
    struct Tok {
        int kind;  // 0 number, 1 name, 2 operator, 3 end
        std::string s;
        double v;
        size_t pos;
    };
    std::vector<Tok> toks_;
    size_t k_ = 0;
    std::vector<std::string> names_;
    ExProgram prog_;
    int depth_ = 0;

    static std::string trim(const std::string &s) {
        size_t b = s.find_first_not_of(" \t\r\n"), e = s.find_last_not_of(" \t\r\n");
        return b == std::string::npos ? std::string() : s.substr(b, e - b + 1);
    }
    static int var_index(const std::string &s) {
        static const char *v[kExVars] = {"x0", "y0", "z0", "x", "y", "z", "ux", "uy", "uz", "t", "dt", "dx"};
        for (int q = 0; q < kExVars; q++)
            if (s == v[q]) return q;
        return -1;
    }
    static int fn_index(const std::string &s) {
        static const char *f[EXF_NUM] = {"sin", "cos", "tan", "cot", "sinh", "cosh", "tanh", "coth", "sqrt", "abs",
                                         "log", "ln"};
        for (int q = 0; q < EXF_NUM; q++)
            if (s == f[q]) return q;
        return -1;
    }
    static bool reserved(const std::string &s) {
        return s == "and" || s == "or" || s == "if" || s == "skip" || s == "Skip" || s == "pow" || var_index(s) >= 0 ||
               fn_index(s) >= 0;
    }
    static bool valid_local(const std::string &s) {
        if (s.empty() || !(std::isalpha((unsigned char)s[0]) || s[0] == '_')) return false;
        for (char ch : s)
            if (!(std::isalnum((unsigned char)ch) || ch == '_')) return false;
        return !reserved(s);
    }

    [[noreturn]] void fail(const std::string &what, size_t pos) {
        throw std::runtime_error(what + " at position " + std::to_string(pos) + " of the " + ctx_);
    }
    std::string ctx_;

    void tokenize(const std::string &src) {
        toks_.clear();
        size_t i = 0;
        const size_t n = src.size();
        while (true) {
            while (i < n && std::isspace((unsigned char)src[i])) i++;
            if (i >= n) break;
            const char ch = src[i];
            if (std::isdigit((unsigned char)ch) || (ch == '.' && i + 1 < n && std::isdigit((unsigned char)src[i + 1]))) {
                size_t j = i;
                while (j < n && std::isdigit((unsigned char)src[j])) j++;
                if (j < n && src[j] == '.') {
                    j++;
                    while (j < n && std::isdigit((unsigned char)src[j])) j++;
                }
                if (j < n && (src[j] == 'e' || src[j] == 'E')) {
                    size_t q = j + 1;
                    if (q < n && (src[q] == '+' || src[q] == '-')) q++;
                    if (q < n && std::isdigit((unsigned char)src[q])) {
                        while (q < n && std::isdigit((unsigned char)src[q])) q++;
                        j = q;
                    }
                }
                const std::string num = src.substr(i, j - i);
                toks_.push_back({0, num, std::strtod(num.c_str(), nullptr), i});
                i = j;
            } else if (std::isalpha((unsigned char)ch) || ch == '_') {
                size_t j = i;
                while (j < n && (std::isalnum((unsigned char)src[j]) || src[j] == '_')) j++;
                toks_.push_back({1, src.substr(i, j - i), 0.0, i});
                i = j;
            } else {
                static const char *two[] = {"<=", ">=", "==", "!="};
                bool matched = false;
                for (const char *t : two)
                    if (src.compare(i, 2, t) == 0) {
                        toks_.push_back({2, t, 0.0, i});
                        i += 2;
                        matched = true;
                        break;
                    }
                if (matched) continue;
                if (std::string("+-*/^<>(),").find(ch) == std::string::npos)
                    fail(std::string("unexpected character '") + ch + "'", i);
                toks_.push_back({2, std::string(1, ch), 0.0, i});
                i++;
            }
        }
        toks_.push_back({3, "", 0.0, n});
        k_ = 0;
    }

    const Tok &peek() const { return toks_[k_]; }
    bool is_op(const char *s) const { return peek().kind == 2 && peek().s == s; }
    bool is_name(const char *s) const { return peek().kind == 1 && peek().s == s; }
    void expect_op(const char *s) {
        if (!is_op(s)) fail(std::string("expected '") + s + "'", peek().pos);
        k_++;
    }

    void emit(uint8_t op, uint8_t a, int b, int stack_change) {
        if (prog_.code.size() >= 65000) throw std::runtime_error("expression too long");
        prog_.code.push_back(ExInstr{op, a, (uint16_t)b});
        depth_ += stack_change;
        if (depth_ > prog_.max_stack) prog_.max_stack = depth_;
        if (depth_ > kExMaxStack) throw std::runtime_error("expression nests too deeply");
    }
    void emit_const(double v) {
        if (prog_.consts.size() >= 65000) throw std::runtime_error("too many constants");
        prog_.consts.push_back(v);
        emit(EX_CONST, 0, (int)prog_.consts.size() - 1, +1);
    }

    void parse_all(const std::string &src, const std::string &what) {
        ctx_ = what;
        tokenize(src);
        if (peek().kind == 3) fail("empty", 0);
        or_expr();
        if (peek().kind != 3) fail("unexpected '" + peek().s + "'", peek().pos);
    }
    void or_expr() {
        and_expr();
        while (is_name("or")) {
            k_++;
            and_expr();
            emit(EX_OR, 0, 0, -1);
        }
    }
    void and_expr() {
        cmp_expr();
        while (is_name("and")) {
            k_++;
            cmp_expr();
            emit(EX_AND, 0, 0, -1);
        }
    }
    void cmp_expr() {
        add_expr();
        while (true) {
            uint8_t op;
            if (is_op("<")) op = EX_LT;
            else if (is_op(">")) op = EX_GT;
            else if (is_op("<=")) op = EX_LE;
            else if (is_op(">=")) op = EX_GE;
            else if (is_op("==")) op = EX_EQ;
            else if (is_op("!=")) op = EX_NE;
            else break;
            k_++;
            add_expr();
            emit(op, 0, 0, -1);
        }
    }
    void add_expr() {
        mul_expr();
        while (is_op("+") || is_op("-")) {
            const uint8_t op = is_op("+") ? EX_ADD : EX_SUB;
            k_++;
            mul_expr();
            emit(op, 0, 0, -1);
        }
    }
    void mul_expr() {
        unary();
        while (is_op("*") || is_op("/")) {
            const uint8_t op = is_op("*") ? EX_MUL : EX_DIV;
            k_++;
            unary();
            emit(op, 0, 0, -1);
        }
    }
    void unary() {
        if (is_op("-")) {
            k_++;
            unary();
            emit(EX_NEG, 0, 0, 0);
        } else if (is_op("+")) {
            k_++;
            unary();
        } else {
            power();
        }
    }
    void power() {
        primary();
        if (is_op("^")) {
            k_++;
            unary();  // right-associative, the exponent may carry a sign
            emit(EX_POW, 0, 0, -1);
        }
    }
    void primary() {
        const Tok t = peek();
        if (t.kind == 0) {
            k_++;
            emit_const(t.v);
            return;
        }
        if (t.kind == 2 && t.s == "(") {
            k_++;
            or_expr();
            expect_op(")");
            return;
        }
        if (t.kind != 1) fail("unexpected '" + t.s + "'", t.pos);
        k_++;
        if (t.s == "skip" || t.s == "Skip") {
            emit(EX_SKIP, 0, 0, +1);
            return;
        }
        if (t.s == "if") {
            expect_op("(");
            or_expr();
            expect_op(",");
            const size_t jz = prog_.code.size();
            emit(EX_JZ, 0, 0, -1);
            const int d0 = depth_;
            or_expr();
            expect_op(",");
            const size_t jmp = prog_.code.size();
            emit(EX_JMP, 0, 0, 0);
            prog_.code[jz].b = (uint16_t)prog_.code.size();
            depth_ = d0;
            or_expr();
            expect_op(")");
            prog_.code[jmp].b = (uint16_t)prog_.code.size();
            return;
        }
        const int f = fn_index(t.s);
        if (f >= 0 || t.s == "pow") {
            expect_op("(");
            or_expr();
            int nargs = 1;
            while (is_op(",")) {
                k_++;
                or_expr();
                nargs++;
            }
            expect_op(")");
            const int want = f >= 0 ? 1 : 2;
            if (nargs != want)
                fail(t.s + " takes " + std::to_string(want) + " argument(s), got " + std::to_string(nargs), t.pos);
            if (f >= 0) emit(EX_FN, (uint8_t)f, 0, 0);
            else emit(EX_POW, 0, 0, -1);
            return;
        }
        for (size_t q = 0; q < names_.size(); q++)
            if (names_[q] == t.s) {
                emit(EX_LOAD, (uint8_t)q, 0, +1);
                return;
            }
        const int v = var_index(t.s);
        if (v >= 0) {
            emit(EX_VAR, (uint8_t)v, 0, +1);
            return;
        }
        fail("unknown name '" + t.s + "'", t.pos);
    }
};

}  // namespace tl
