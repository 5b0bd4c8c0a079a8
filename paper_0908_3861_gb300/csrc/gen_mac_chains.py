"""Writes the carry-chained multiply-accumulate routines of abf_internal.cuh.

acc (W 32-bit words) += a (W words) * w (B words) modulo 2^(32 W), as PTX
mad/madc chains: for every weight word j, one chain adds the low half of
a_0 w_j at word j and the high halves of a_i w_j at words j+1+i, a second
chain adds the low halves of a_i w_j (i >= 1) at words j+i; each chain
carries up to the top word, and the carry out of the top is the modulus.
Running it prints the routines and checks the schedule against Python
integers (the carry semantics of mad.cc / madc) on random operands; the
build (build.py) runs check_header() first, which repeats that check and
requires abf_internal.cuh to hold exactly the routines generated here.
"""
def chain(W, B):
    lines = []
    # operands: r0..r{W-1} = %0..%{W-1}; a0..a{W-1} = %W..%{2W-1}; w0..w{B-1} = %{2W}..
    R = lambda k: '%%%d' % k
    A = lambda i: '%%%d' % (W + i)
    Wd = lambda j: '%%%d' % (2 * W + j)
    for j in range(B):
        if j >= W:
            break
        # chain 1: lo(a0 wj) at j, hi(a_i wj) at j+1+i
        ops = [('lo', 0, j)] + [('hi', i, j + 1 + i) for i in range(W) if j + 1 + i < W]
        for k, (h, i, pos) in enumerate(ops):
            first, last = k == 0, k == len(ops) - 1
            op = ('mad' if first else 'madc') + '.' + h + ('' if last else '.cc') + '.u32'
            lines.append('%-15s %s, %s, %s, %s;' % (op, R(pos), A(i), Wd(j), R(pos)))
        # chain 2: lo(a_i wj) at j+i, i >= 1
        ops = [('lo', i, j + i) for i in range(1, W) if j + i < W]
        for k, (h, i, pos) in enumerate(ops):
            first, last = k == 0, k == len(ops) - 1
            op = ('mad' if first else 'madc') + '.' + h + ('' if last else '.cc') + '.u32'
            lines.append('%-15s %s, %s, %s, %s;' % (op, R(pos), A(i), Wd(j), R(pos)))
    return lines

def emit(W, B, name):
    L = W // 2
    body = chain(W, B)
    out = []
    out.append('// acc += g * w (mod 2^%d): %d-limb g, %d-bit w; %d multiply-adds in carry chains.' % (32 * W, L, 32 * B, len(body)))
    wargs = ', '.join('uint32_t w%d' % j for j in range(B))
    out.append('__device__ __forceinline__ void %s(Wide<%d>& acc, const Wide<%d>& g, %s) {' % (name, L, L, wargs))
    out.append('  uint32_t r[%d], a[%d];' % (W, W))
    out.append('#pragma unroll')
    out.append('  for (int i = 0; i < %d; ++i) {' % L)
    out.append('    r[2 * i] = (uint32_t)acc.w[i]; r[2 * i + 1] = (uint32_t)(acc.w[i] >> 32);')
    out.append('    a[2 * i] = (uint32_t)g.w[i]; a[2 * i + 1] = (uint32_t)(g.w[i] >> 32);')
    out.append('  }')
    out.append('  asm("{\\n\\t"')
    for l in body:
        out.append('      "%s\\n\\t"' % l)
    out.append('      "}"')
    outs = ', '.join('"+r"(r[%d])' % k for k in range(W))
    ins = ', '.join(['"r"(a[%d])' % k for k in range(W)] + ['"r"(w%d)' % j for j in range(B)])
    out.append('      : %s' % outs)
    out.append('      : %s);' % ins)
    out.append('#pragma unroll')
    out.append('  for (int i = 0; i < %d; ++i) acc.w[i] = ((uint64_t)r[2 * i + 1] << 32) | r[2 * i];' % L)
    out.append('}')
    return '\n'.join(out)

ROUTINES = [(6, 2), (8, 2), (4, 4), (6, 4), (8, 4)]


def generate():
    """The routines as they appear in abf_internal.cuh, in order."""
    return [emit(W, B, 'wmac_w%d_b%d' % (W, B)) for (W, B) in ROUTINES]


def sim(W, B, acc, a, w):
    """The chain run on Python integers with the carry semantics of mad.cc /
    madc (the carry flag holds the bit out of the 32-bit sum)."""
    r = [(acc >> (32 * k)) & 0xffffffff for k in range(W)]
    A = [(a >> (32 * k)) & 0xffffffff for k in range(W)]
    Wv = [(w >> (32 * k)) & 0xffffffff for k in range(B)]
    cc = 0
    for l in chain(W, B):
        op, rest = l.split(None, 1)
        d, x, y, _ = [t.strip().strip(';') for t in rest.split(',')]
        di = int(d[1:]); xi = int(x[1:]) - W; yi = int(y[1:]) - 2 * W
        p = A[xi] * Wv[yi]
        part = (p >> 32) if '.hi' in op else (p & 0xffffffff)
        cin = cc if op.startswith('madc') else 0
        s = r[di] + part + cin
        r[di] = s & 0xffffffff
        cc = (s >> 32) if '.cc' in op else 0
    return sum(v << (32 * k) for k, v in enumerate(r))


def verify_schedule(trials=400, seed=0):
    """Every chain schedule equals acc + a w modulo 2^(32 W) on random operands."""
    import random
    rnd = random.Random(seed)
    for (W, B) in [(4, 2), (6, 2), (8, 2), (4, 4), (6, 4), (8, 4), (4, 1), (6, 1), (8, 1)]:
        for _ in range(trials):
            acc = rnd.getrandbits(32 * W); a = rnd.getrandbits(32 * W); w = rnd.getrandbits(32 * B)
            if sim(W, B, acc, a, w) != (acc + a * w) % (1 << (32 * W)):
                raise AssertionError('carry chain schedule wrong for W=%d B=%d' % (W, B))


def check_header(path=None):
    """The build's check: the schedules are right and abf_internal.cuh holds
    exactly the routines this generator writes."""
    import os
    path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), 'abf_internal.cuh')
    verify_schedule()
    with open(path) as fh:
        text = fh.read()
    for body in generate():
        if body not in text:
            raise AssertionError('abf_internal.cuh differs from the generated routine:\n' + body.split('\n')[1])


if __name__ == '__main__':
    import sys
    for body in generate():
        print(body)
        print()
    verify_schedule(trials=2000)
    print('// schedule verified', file=sys.stderr)
