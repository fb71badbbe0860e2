"""The paper's value-count model -- TEST INFRASTRUCTURE ONLY.

Sec. III.B counts the metric values the approach computes for a system of
c classes and m methods:
  * fan-in and fan-out, one value each per method: 2m;
  * similarity, one value per unordered method pair: m(m-1)/2;
  * LCOM, for each class as it is and for each class after receiving each
    method (the worst case of the moves it assesses): c + c m = c(m+1);
  * CBO, the same number as LCOM in the worst case.

    #values = 2m + m(m-1)/2 + 2c(m+1)

Table I prints #values (in millions) for its 13 systems; the golden file
``tests/golden/table1_values.csv`` holds those printed rows, so Table I pins
every term of the sum below.
"""


def fan_values(m: int) -> int:
    """fan-in and fan-out of every method (Sec. III.B, first term)."""
    return 2 * m


def similarity_values(m: int) -> int:
    """one similarity value per unordered pair of methods (Sec. III.B)."""
    return m * (m - 1) // 2


def lcom_values(c: int, m: int) -> int:
    """#LCOM values of Sec. III.B: each class, and each class after a move in."""
    return c + c * m


def cbo_values(c: int, m: int) -> int:
    """#CBO values: as many as the LCOM values in the worst case (Sec. III.B)."""
    return lcom_values(c, m)


def count_values(c: int, m: int) -> int:
    """#values of Sec. III.B: the sum of the four counts above."""
    return fan_values(m) + similarity_values(m) + lcom_values(c, m) + cbo_values(c, m)
