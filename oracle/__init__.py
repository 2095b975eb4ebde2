"""CPU oracle for the m-double matrix product (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline leg
may import, call or execute anything in this package.  The GPU library shares no
code with it: no kernels, headers, helpers, tables or constants.  The oracle's
inputs come from ``synthetic`` (random numbers only) and from nothing computed
on the GPU.

Parts, each a plain and slow restatement of what the paper defines:

* ``exact``    -- exact values of m-doubles as dyadic rationals (Python ints),
                  the exact product C = A B, the componentwise error bound
                  2K 2^(-52m) (|A||B|) and greedy round-to-nearest of an exact
                  value into m nonoverlapping doubles (Section 1 definition of a
                  multiple double: an unevaluated sum of nonoverlapping doubles).
* ``slicing``  -- the error-free summation of Section 2: a shared exponent per
                  row (column), fixed-point pieces with zero high bits, the
                  diagonal sums s_i of Section 2 / Section 4, exact fusion.
                  Bit-exact reference for the GPU digits and integer sums.
* ``crt``      -- the residue form the Ozaki scheme points to (Sections 1 and
                  4): the same fixed-point integers multiplied exactly through
                  residues modulo pairwise coprime moduli and the Chinese
                  remainder theorem, then rounded greedily.
* ``series``   -- products of truncated power series (Section 1's
                  application): every coefficient c_i = sum_{k<=i} a_k b_{i-k}
                  exactly, its bound, and its error-free summation.
* ``textbook`` -- the "ordinary" m-double product of Table 2: multiply-add in
                  m-double arithmetic with two-sum and Dekker two-product, in C
                  (``textbook.c``) for timing and in Python for operation counts
                  (Table 1).
"""
