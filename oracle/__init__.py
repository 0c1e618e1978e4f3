"""CPU oracle for the Tensor Data Platform hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import, call, link or execute
anything in this package.  The product path (``paper_2211_02753_b300``)
never imports it, and this package never imports the product path; the two
share no code.  The only common dependency is ``gen`` (seeded inputs, no
method arithmetic).

Modules:
  relational -- exact int64 filter / group-by / join / top-k / sort (plain C,
                ``oracle.c``, loaded through ctypes).
  brute      -- pure-Python nested-loop / dict versions for tiny tables, used
                to pin ``relational``.
  soft       -- fp64 soft filter, soft aggregation and their adjoints (Sec. 4),
                soft group-by on probability-encoded columns.
  cnn        -- fp64 glyph CNN forward/backward, the trainable query loss and
                Adam (Sec. 3 training loop); the two-head Digit x Size query.
  dictionary -- order-preserving dictionary codes of string columns.
  llp        -- fp64 learning from label proportions (Sec. 5.3) and its
                label-DP variant (Sec. 5.4).
  softsort   -- fp64 soft ORDER BY ... LIMIT k: logistic soft ranks, soft
                top-k membership and sum, their adjoints; the exact ranks.
"""
