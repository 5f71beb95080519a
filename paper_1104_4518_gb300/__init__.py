"""GB300 breadth-first search (placeholder; the binding is added with the library)."""
