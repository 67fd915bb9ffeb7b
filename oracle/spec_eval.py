"""Plain FP64 evaluation of a sequence program (the statement language of
the paper's compiler input, Section II and Fig. 1: declarations, then
assignments of linear-algebra expressions).

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import this module; the library's product
path never does.

Each statement is evaluated in order on whole numpy arrays: vectors are
column arrays of shape (n, 1), `'` transposes, `*` is the matrix product
when both operands are arrays and scaling otherwise.  There is no fusion
and no partitioning: this is the definition the generated passes must
reproduce.  Storage order (`matrix(row)`) does not change the values, so it
is ignored here.  The parser (a shunting-yard over a character scanner) is
written for this evaluator alone.
"""
import numpy as np

_PREC = {"+": 1, "-": 1, "*": 2, "neg": 3}


def _scan(text):
    toks, i = [], 0
    while i < len(text):
        c = text[i]
        if c.isspace():
            i += 1
        elif c.isalpha() or c == "_":
            j = i
            while j < len(text) and (text[j].isalnum() or text[j] == "_"):
                j += 1
            toks.append(("id", text[i:j]))
            i = j
        elif c.isdigit() or c == ".":
            j = i
            while j < len(text) and (text[j].isdigit() or text[j] in ".eE" or
                                     (text[j] in "+-" and text[j - 1] in "eE")):
                j += 1
            toks.append(("num", float(text[i:j])))
            i = j
        elif c in "+-*()'":
            toks.append(("op", c))
            i += 1
        else:
            raise ValueError("bad character %r" % c)
    return toks


def _rpn(toks):
    """Operator-precedence conversion to postfix; '-' after an operator or
    at the start is negation; "'" applies at once to the operand before it."""
    out, stack, prev_operand = [], [], False
    for kind, v in toks:
        if kind in ("id", "num"):
            out.append((kind, v))
            prev_operand = True
        elif v == "'":
            out.append(("op", "'"))
        elif v == "(":
            stack.append(v)
            prev_operand = False
        elif v == ")":
            while stack and stack[-1] != "(":
                out.append(("op", stack.pop()))
            if not stack:
                raise ValueError("unbalanced parentheses")
            stack.pop()
            prev_operand = True
        else:
            op = v if (prev_operand or v != "-") else "neg"
            if op == "neg":
                stack.append(op)
            else:
                while stack and stack[-1] != "(" and _PREC[stack[-1]] >= _PREC[op]:
                    out.append(("op", stack.pop()))
                stack.append(op)
            prev_operand = False
    while stack:
        op = stack.pop()
        if op == "(":
            raise ValueError("unbalanced parentheses")
        out.append(("op", op))
    return out


def _apply(op, a, b=None):
    if op == "'":
        return a.T if isinstance(a, np.ndarray) else a
    if op == "neg":
        return -a
    if op == "+":
        return a + b
    if op == "-":
        return a - b
    if isinstance(a, np.ndarray) and isinstance(b, np.ndarray):
        return a @ b
    return a * b


def _kinds(text):
    """{name: 'vector' | 'matrix' | 'scalar'} from the in: and out: lines."""
    kinds = {}
    for raw in text.splitlines():
        line = raw.split("#", 1)[0].strip()
        if not line.lower().startswith(("in:", "out:")):
            continue
        for entry in line.split(":", 1)[1].split(","):
            if ":" in entry:
                names, ty = entry.split(":", 1)
                for k in ("vector", "matrix", "scalar"):
                    if ty.strip().lower().startswith(k):
                        kinds.update((n, k) for n in names.split())
    return kinds


def evaluate(text, inputs):
    """Runs the program on `inputs` ({name: float, 1-D vector or 2-D
    matrix}); returns {name: value} for every assigned name (vectors 1-D)."""
    env = {}
    for k, v in inputs.items():
        if isinstance(v, np.ndarray):
            v = np.asarray(v, dtype=np.float64)
            env[k] = v.reshape(-1, 1) if v.ndim == 1 else v
        else:
            env[k] = float(v)
    # A declared vector is returned 1-D and a declared matrix 2-D, whatever
    # their sizes; an undeclared (temporary) result by its shape.
    kinds = _kinds(text)
    assigned = {}
    for raw in text.splitlines():
        line = raw.split("#", 1)[0].strip().strip("{}").strip()
        if "=" not in line or line.lower().startswith(("in:", "out:")):
            continue
        tgt, rhs = (s.strip() for s in line.split("=", 1))
        stack = []
        for kind, v in _rpn(_scan(rhs)):
            if kind == "num":
                stack.append(v)
            elif kind == "id":
                stack.append(env[v])
            elif v in ("'", "neg"):
                stack.append(_apply(v, stack.pop()))
            else:
                b = stack.pop()
                a = stack.pop()
                stack.append(_apply(v, a, b))
        if len(stack) != 1:
            raise ValueError("malformed expression %r" % rhs)
        env[tgt] = stack[0]
        val = stack[0]
        is_vec = kinds.get(tgt) == "vector" or (tgt not in kinds and isinstance(val, np.ndarray) and
                                               val.shape[1:] == (1,))
        assigned[tgt] = val.reshape(-1) if isinstance(val, np.ndarray) and is_vec else val
    return assigned
